// k_particles.cu -- the per-particle passes of the fastdf method (Elbers 2022):
//   initial: the pre-initial momentum transform (eq:transform, Sec. 2.1);
//   push:    one leapfrog pass of the separable equations of motion
//            (eq:releq_approx, eq:geodesic_approx, Sec. 3.3): drift by the
//            exact free-streaming integral for frozen q, periodic wrap,
//            trilinear gather of the gradient grid, kick;
//   export:  positions, momenta and delta-f weights w = 1 - fbar(q)/fbar(p)
//            (Sec. 2.2) in particle-index order;
//   deposit: the weighted CIC density estimate (eq:empirical_rho).
//
// Three state forms.  The plain form keeps x, q, q_0 in FP64 and reads an FP64
// grid.  The FP64-state form (the FP32/BF16-grid precision settings) keeps x and q
// in FP64 and q_0 in FP32, reads an FP32 or BF16 grid, and spends as few FP64
// instructions as FP64 integrals allow (k_push_wide).  The split-state form keeps
// positions as 32-bit fixed-point fractions of the box (the periodic wrap is the
// integer overflow), momenta as q = q_0 + dq with both parts in FP32, and evaluates
// the drift integral in float-float so that no FP64 instruction runs in its pass.
#include <cuda_bf16.h>

#include <type_traits>
#include <utility>

#include "device_math.cuh"

namespace fdf {

namespace {

constexpr int kThreads = 256;

unsigned grid_for(int64_t n, int per_sm = 16)
{
    int64_t b = (n + kThreads - 1) / kThreads;
    const int64_t cap = 152LL * per_sm;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

// The particle passes launch at the device's greatest execution priority
// (cudaLaunchAttributePriority).  The grids of the next pass are built on another
// stream at the default priority; when both wait for room on the SMs, the block
// scheduler places the pass's blocks first.
int pass_priority()
{
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) return 0;
    return greatest;
}

// A launch error is left for the caller's cudaGetLastError.
template <typename... K, typename... A>
void launch_pass(void (*kernel)(K...), unsigned blocks, cudaStream_t s, A&&... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributePriority;
    at[0].val.priority = pass_priority();
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

// ---- grid reads ------------------------------------------------------------
template <typename Gt> struct Cell;
template <> struct Cell<float> {
    // one 256-bit load per cell (a cell's 8 slots are 32 contiguous, 32-byte aligned bytes);
    // not allocated in L1: the loads that would hit are too few to pay for the fills
    __device__ static void load(const float* G, uint32_t c, float v[8])
    {
        const float* g = G + 8 * (size_t)c;
        asm("ld.global.nc.L1::no_allocate.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
            : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
            : "l"(g));
    }
};
template <> struct Cell<__nv_bfloat16> {
    __device__ static void load(const __nv_bfloat16* G, uint32_t c, float v[8])
    {
        uint4 u;
        asm("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
            : "=r"(u.x), "=r"(u.y), "=r"(u.z), "=r"(u.w)
            : "l"(reinterpret_cast<const uint4*>(G) + c));
        const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[2 * k] = __uint_as_float(w[k] << 16);
            v[2 * k + 1] = __uint_as_float(w[k] & 0xFFFF0000u);
        }
    }
};

// Trilinear (order r = 1, Sec. 4) read of the 8 slots at a fixed-point position.
template <typename Gt>
__device__ __forceinline__ void gather_fixed(const Gt* __restrict__ G, uint32_t N, uint32_t X0, uint32_t X1,
                                             uint32_t X2, float g[8])
{
    uint32_t ix[2], iy[2], iz[2];
    float fx, fy, fz;
    fixed_cell(X0, N, ix[0], ix[1], fx);
    fixed_cell(X1, N, iy[0], iy[1], fy);
    fixed_cell(X2, N, iz[0], iz[1], fz);
#pragma unroll
    for (int s = 0; s < 8; ++s) g[s] = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int cx = c & 1, cy = (c >> 1) & 1, cz = c >> 2;
        const float w = (cx ? fx : 1.f - fx) * (cy ? fy : 1.f - fy) * (cz ? fz : 1.f - fz);
        float v[8];
        Cell<Gt>::load(G, (iz[cz] * N + iy[cy]) * N + ix[cx], v);
#pragma unroll
        for (int s = 0; s < 8; ++s) g[s] = fmaf(w, v[s], g[s]);
    }
}

// One axis of the order-2 kernel (Sec. 4, r = 2: the quadratic B-spline, or
// triangular-shaped cloud) from a coordinate's cell i0, next node i1 and fraction f:
// the nearest node c and its neighbours, with d = u - c in [-1/2, 1/2) and weights
// (1/2 - d)^2/2, 3/4 - d^2, (1/2 + d)^2/2.
__device__ __forceinline__ void tsc_from_cell(uint32_t i0, uint32_t i1, float f, uint32_t N, uint32_t idx[3],
                                              float w[3])
{
    const bool up = f >= 0.5f;
    const uint32_t c = up ? i1 : i0;
    const float d = up ? f - 1.f : f;
    idx[0] = c == 0u ? N - 1u : c - 1u;
    idx[1] = c;
    idx[2] = c + 1u == N ? 0u : c + 1u;
    const float l = 0.5f - d, r = 0.5f + d;
    w[0] = 0.5f * l * l;
    w[1] = 0.75f - d * d;
    w[2] = 0.5f * r * r;
}

// The same at a fixed-point coordinate.
__device__ __forceinline__ void tsc_axis(uint32_t X, uint32_t N, uint32_t idx[3], float w[3])
{
    uint32_t i0, i1;
    float f;
    fixed_cell(X, N, i0, i1, f);
    tsc_from_cell(i0, i1, f, N, idx, w);
}

template <typename Gt>
__device__ __forceinline__ void gather_fixed_tsc(const Gt* __restrict__ G, uint32_t N, uint32_t X0, uint32_t X1,
                                                 uint32_t X2, float g[8])
{
    uint32_t ix[3], iy[3], iz[3];
    float wx[3], wy[3], wz[3];
    tsc_axis(X0, N, ix, wx);
    tsc_axis(X1, N, iy, wy);
    tsc_axis(X2, N, iz, wz);
#pragma unroll
    for (int s = 0; s < 8; ++s) g[s] = 0.f;
#pragma unroll 1
    for (int cz = 0; cz < 3; ++cz) {
#pragma unroll
        for (int cy = 0; cy < 3; ++cy) {
            const uint32_t row = (iz[cz] * N + iy[cy]) * N;
            const float wzy = wz[cz] * wy[cy];
#pragma unroll
            for (int cx = 0; cx < 3; ++cx) {
                const float w = wx[cx] * wzy;
                float v[8];
                Cell<Gt>::load(G, row + ix[cx], v);
#pragma unroll
                for (int s = 0; s < 8; ++s) g[s] = fmaf(w, v[s], g[s]);
            }
        }
    }
}

// The kernel of order r (1 or 2) at a fixed-point position.
template <typename Gt>
__device__ __forceinline__ void gather_order(int order, const Gt* __restrict__ G, uint32_t N, uint32_t X0,
                                             uint32_t X1, uint32_t X2, float g[8])
{
    if (order == 2) gather_fixed_tsc<Gt>(G, N, X0, X1, X2, g);
    else gather_fixed<Gt>(G, N, X0, X1, X2, g);
}

// ---- reads of an FP32 or BF16 grid at an FP64 position (the FP64-state form) ----
// The position goes to FP32 on the integer pipe; u = x N / L in FP32 then locates the
// cell to ~2^-24 N of a cell, far below what moves a trilinear read of the fields.
__device__ __forceinline__ void float_cell(double x, float invh, uint32_t N, uint32_t& i0, uint32_t& i1, float& f)
{
    const float u = d2f_bits(x) * invh;       // x in [0, L): u in [0, N]
    uint32_t i = (uint32_t)u;
    f = u - (float)i;
    i = i >= N ? i - N : i;                    // u rounded up to N: node 0
    i = i < N ? i : N - 1u;                    // (never taken for x in [0, L); keeps reads in the grid)
    i0 = i;
    i1 = i + 1u == N ? 0u : i + 1u;
}

template <typename Gt>
__device__ __forceinline__ void gather_wide(int order, const Gt* __restrict__ G, uint32_t N, float invh,
                                            const double x[3], float g[8])
{
    uint32_t ix[3], iy[3], iz[3];
    float wx[3], wy[3], wz[3];
    uint32_t i0, i1;
    float f;
#pragma unroll
    for (int s = 0; s < 8; ++s) g[s] = 0.f;
    if (order == 2) {
        float_cell(x[0], invh, N, i0, i1, f);
        tsc_from_cell(i0, i1, f, N, ix, wx);
        float_cell(x[1], invh, N, i0, i1, f);
        tsc_from_cell(i0, i1, f, N, iy, wy);
        float_cell(x[2], invh, N, i0, i1, f);
        tsc_from_cell(i0, i1, f, N, iz, wz);
#pragma unroll 1
        for (int cz = 0; cz < 3; ++cz) {
#pragma unroll
            for (int cy = 0; cy < 3; ++cy) {
                const uint32_t row = (iz[cz] * N + iy[cy]) * N;
                const float wzy = wz[cz] * wy[cy];
#pragma unroll
                for (int cx = 0; cx < 3; ++cx) {
                    const float w = wx[cx] * wzy;
                    float v[8];
                    Cell<Gt>::load(G, row + ix[cx], v);
#pragma unroll
                    for (int s = 0; s < 8; ++s) g[s] = fmaf(w, v[s], g[s]);
                }
            }
        }
        return;
    }
    float fx, fy, fz;
    float_cell(x[0], invh, N, ix[0], ix[1], fx);
    float_cell(x[1], invh, N, iy[0], iy[1], fy);
    float_cell(x[2], invh, N, iz[0], iz[1], fz);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int cx = c & 1, cy = (c >> 1) & 1, cz = c >> 2;
        const float w = (cx ? fx : 1.f - fx) * (cy ? fy : 1.f - fy) * (cz ? fz : 1.f - fz);
        float v[8];
        Cell<Gt>::load(G, (iz[cz] * N + iy[cy]) * N + ix[cx], v);
#pragma unroll
        for (int s = 0; s < 8; ++s) g[s] = fmaf(w, v[s], g[s]);
    }
}

// FP64 read at an FP64 position in [0, L).
__device__ __forceinline__ void gather_f64(const double* __restrict__ G, int N, double invh, const double x[3],
                                           double g[8])
{
    int i0[3], i1[3];
    double f[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double u = x[d] * invh;
        const double fl = floor(u);
        f[d] = u - fl;
        int i = (int)fl;
        if (i >= N) i -= N;
        if (i < 0) i += N;
        i0[d] = i;
        i1[d] = i + 1 == N ? 0 : i + 1;
    }
#pragma unroll
    for (int s = 0; s < 8; ++s) g[s] = 0.0;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int cx = c & 1, cy = (c >> 1) & 1, cz = c >> 2;
        const double w = (cx ? f[0] : 1.0 - f[0]) * (cy ? f[1] : 1.0 - f[1]) * (cz ? f[2] : 1.0 - f[2]);
        const size_t cell = ((size_t)(cz ? i1[2] : i0[2]) * N + (cy ? i1[1] : i0[1])) * N + (cx ? i1[0] : i0[0]);
        const double2* p = reinterpret_cast<const double2*>(G) + 4 * cell;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const double2 v = __ldg(p + k);
            g[2 * k] += w * v.x;
            g[2 * k + 1] += w * v.y;
        }
    }
}

// FP64 order-2 read at an FP64 position in [0, L).
__device__ __forceinline__ void gather_f64_tsc(const double* __restrict__ G, int N, double invh, const double x[3],
                                               double g[8])
{
    int idx[3][3];
    double w[3][3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double u = x[d] * invh;
        const double c = floor(u + 0.5);
        const double e = u - c;
        int i = (int)c;
        if (i >= N) i -= N;
        if (i < 0) i += N;
        idx[d][0] = i == 0 ? N - 1 : i - 1;
        idx[d][1] = i;
        idx[d][2] = i + 1 == N ? 0 : i + 1;
        w[d][0] = 0.5 * (0.5 - e) * (0.5 - e);
        w[d][1] = 0.75 - e * e;
        w[d][2] = 0.5 * (0.5 + e) * (0.5 + e);
    }
#pragma unroll
    for (int s = 0; s < 8; ++s) g[s] = 0.0;
    for (int cz = 0; cz < 3; ++cz)
        for (int cy = 0; cy < 3; ++cy)
            for (int cx = 0; cx < 3; ++cx) {
                const double wt = w[0][cx] * w[1][cy] * w[2][cz];
                const size_t cell = ((size_t)idx[2][cz] * N + idx[1][cy]) * N + idx[0][cx];
                const double2* p = reinterpret_cast<const double2*>(G) + 4 * cell;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const double2 v = __ldg(p + k);
                    g[2 * k] += wt * v.x;
                    g[2 * k + 1] += wt * v.y;
                }
            }
}

__device__ __forceinline__ void gather_f64_order(int order, const double* __restrict__ G, int N, double invh,
                                                 const double x[3], double g[8])
{
    if (order == 2) gather_f64_tsc(G, N, invh, x, g);
    else gather_f64(G, N, invh, x, g);
}

__device__ __forceinline__ double wrap_f64(double x, double L, double invL)
{
    double y = x - L * floor(x * invL);
    if (y < 0.0) y += L;
    if (y >= L) y -= L;
    return y;
}

// Round a float-float count of position quanta to the nearest integer, modulo
// 2^32.  A hi part beyond +-2^31 is a multiple of 256 and is first reduced by an
// exact multiple of 2^32; what remains converts to int32 exactly, and the
// fractional part of hi plus lo adds the last quanta.
__device__ __forceinline__ uint32_t round_mod32(FF d)
{
    float h = d.hi;
    if (fabsf(h) >= 2147483648.f)
        h = __fsub_rn(h, __fmul_rn(4294967296.f, rintf(__fmul_rn(h, 2.3283064365386963e-10f))));
    const int i = __float2int_rn(h);
    const int i2 = __float2int_rn(__fadd_rn(__fsub_rn(h, (float)i), d.lo));
    return (uint32_t)i + (uint32_t)i2;
}

struct Masses {
    double m[kMaxSpecies];
};

// ---- initial transform -----------------------------------------------------
// q_i <- q_i (1 - psi/2) - (eps tau_0 / 6) d_i psi  (eq:transform with delta = -2 psi,
// theta = k^2 tau psi / 2, nu = 4, omega = 4/3), eps = sqrt(p^2 + m^2 a_0^2).
// F: the state form (kPlain, kWide, kFixed).  The transform reads the fields at the
// sampled fixed-point positions in every form.
template <int F, typename Gt>
__global__ void __launch_bounds__(kThreads) k_initial(ParticleState st, int64_t n, int64_t n_part, Masses ms,
                                                      double a0, double tau0, int order, int N, double L,
                                                      const Gt* __restrict__ G)
{
    const double tau0_6 = tau0 / 6.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double m = ms.m[i / n_part];
        const uint32_t X0 = st.X[i], X1 = st.X[n + i], X2 = st.X[2 * n + i];
        double g[8];
        double x[3];
        x[0] = L * ((double)X0 * 2.3283064365386963e-10);
        x[1] = L * ((double)X1 * 2.3283064365386963e-10);
        x[2] = L * ((double)X2 * 2.3283064365386963e-10);
        if constexpr (F == kPlain) {
            gather_f64_order(order, reinterpret_cast<const double*>(G), N, (double)N / L, x, g);
        } else {
            float gf[8];
            gather_order<Gt>(order, G, (uint32_t)N, X0, X1, X2, gf);
#pragma unroll
            for (int s = 0; s < 8; ++s) g[s] = (double)gf[s];
        }
        const double p = st.pmag[i];
        const double eps = sqrt(p * p + m * m * a0 * a0);
        const double c = eps * tau0_6;          // eps tau0 / 6 (tau0/6 formed once)
        const double r = 1.0 - 0.5 * g[7];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double q = st.qs[d * n + i] * r - c * g[d];
            if constexpr (F == kPlain) {
                st.xd[d * n + i] = x[d];
                st.qd[d * n + i] = q;
                st.q0d[d * n + i] = q;
            } else if constexpr (F == kWide) {
                st.xd[d * n + i] = x[d];
                st.qd[d * n + i] = q;
                st.q0f[d * n + i] = (float)q;     // q_0 of the kick, stored in FP32
            } else {
                const float hi = (float)q;
                st.q0f[d * n + i] = hi;
                st.dqf[d * n + i] = (float)(q - (double)hi);
            }
        }
    }
}

// ---- the fused leapfrog pass, split form -------------------------------------
// A pass advances every particle through a.nsub sub-steps (temporal blocking): the
// particle's state is read once, carried through the sub-steps in registers and
// written once; each sub-step's kick reads its own grid.  The arithmetic of a
// sub-step does not depend on how the steps are grouped into passes.
__device__ __forceinline__ int species_of(const PushArgs& a, int64_t i)
{
    return (int)(i >= a.sp_begin[0]) + (int)(i >= a.sp_begin[1]) + (int)(i >= a.sp_begin[2]);
}

struct SplitState {
    uint32_t X0, X1, X2;
    float qa, qb, qc, da, db, dc;
};

__device__ __forceinline__ SplitState load_split(const uint32_t* __restrict__ X, const float* __restrict__ q0f,
                                                 const float* __restrict__ dqf, int64_t n, int64_t i)
{
    SplitState s;
    s.X0 = __ldcs(X + i);
    s.X1 = __ldcs(X + n + i);
    s.X2 = __ldcs(X + 2 * n + i);
    s.qa = __ldcs(q0f + i);
    s.qb = __ldcs(q0f + n + i);
    s.qc = __ldcs(q0f + 2 * n + i);
    s.da = __ldcs(dqf + i);
    s.db = __ldcs(dqf + n + i);
    s.dc = __ldcs(dqf + 2 * n + i);
    return s;
}

// ---- the gather from a shared-memory tile of the grid (split-state pass) ---------------
// The particles are sorted by cell, so the 256 particles of a block sit in a few
// neighbouring buckets.  Per kick, the block loads the grid cells of the box that holds
// every particle's cell and its upper neighbours once into shared memory, and each
// particle reads its eight corners there instead of from L2.  The box is taken about the
// block's first particle (minimum image on the periodic grid); one larger than
// kTileCells, or a call that is not of order 1, returns false and the caller reads G
// directly.  Every thread of the block calls it (it synchronises the block); `live`
// marks the threads with a particle.
constexpr int kTileCells = 640;

template <typename Gt> struct TileRec;
template <> struct TileRec<float> { static constexpr int kWords = 2; };          // 32-byte records
template <> struct TileRec<__nv_bfloat16> { static constexpr int kWords = 1; };  // 16-byte records

struct TileShared {
    uint4 rec[kTileCells * 2];
    int ref[3];
    int box[6];      // lo x, y, z, extent x, y, z (cells)
    int red[kThreads / 32][6];
};

template <typename Gt>
__device__ __forceinline__ void tile_unpack(const uint4* r, float v[8])
{
    if constexpr (TileRec<Gt>::kWords == 2) {
        const uint32_t w[8] = {r[0].x, r[0].y, r[0].z, r[0].w, r[1].x, r[1].y, r[1].z, r[1].w};
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = __uint_as_float(w[k]);
    } else {
        const uint32_t w[4] = {r[0].x, r[0].y, r[0].z, r[0].w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[2 * k] = __uint_as_float(w[k] << 16);
            v[2 * k + 1] = __uint_as_float(w[k] & 0xFFFF0000u);
        }
    }
}

template <typename Gt>
__device__ bool tile_gather(TileShared& sh, const Gt* __restrict__ G, uint32_t N, bool live, uint32_t X0, uint32_t X1,
                            uint32_t X2, float g[8])
{
    constexpr int W = TileRec<Gt>::kWords;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t c[3] = {__umulhi(X0, N), __umulhi(X1, N), __umulhi(X2, N)};
    if (tid == 0) {
#pragma unroll
        for (int k = 0; k < 3; ++k) sh.ref[k] = (int)c[k];
    }
    __syncthreads();
    const int half = (int)(N >> 1), mask = (int)N - 1;
    int d[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) d[k] = live ? (((int)c[k] - sh.ref[k] + half) & mask) - half : 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int mn = __reduce_min_sync(0xffffffffu, d[k]);
        const int mx = __reduce_max_sync(0xffffffffu, d[k]);
        if (lane == 0) {
            sh.red[warp][k] = mn;
            sh.red[warp][3 + k] = mx;
        }
    }
    __syncthreads();
    if (tid == 0) {
        int lo[3], hi[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            lo[k] = sh.red[0][k];
            hi[k] = sh.red[0][3 + k];
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
                lo[k] = min(lo[k], sh.red[w][k]);
                hi[k] = max(hi[k], sh.red[w][3 + k]);
            }
            sh.box[k] = lo[k];
            sh.box[3 + k] = hi[k] - lo[k] + 2;      // the cells and their upper neighbours
        }
    }
    __syncthreads();
    const int ex = sh.box[3], ey = sh.box[4], ez = sh.box[5];
    const int vol = ex * ey * ez;
    if (vol > kTileCells || ex > (int)N || ey > (int)N || ez > (int)N) return false;   // block-uniform
    const int bx = sh.ref[0] + sh.box[0], by = sh.ref[1] + sh.box[1], bz = sh.ref[2] + sh.box[2];
    for (int t = tid; t < vol; t += blockDim.x) {
        const int ax = t % ex, ay = (t / ex) % ey, az = t / (ex * ey);
        const uint32_t cell = ((uint32_t)((bz + az) & mask) * N + (uint32_t)((by + ay) & mask)) * N +
                              (uint32_t)((bx + ax) & mask);
        const uint4* src = reinterpret_cast<const uint4*>(G) + (size_t)cell * W;
#pragma unroll
        for (int w = 0; w < W; ++w) sh.rec[t * W + w] = __ldg(src + w);
    }
    __syncthreads();
    if (live) {
        uint32_t i0, i1;
        float f[3];
        int l[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const uint32_t Xk = k == 0 ? X0 : (k == 1 ? X1 : X2);
            fixed_cell(Xk, N, i0, i1, f[k]);
            l[k] = d[k] - sh.box[k];
        }
#pragma unroll
        for (int s = 0; s < 8; ++s) g[s] = 0.f;
#pragma unroll
        for (int cn = 0; cn < 8; ++cn) {
            const int cx = cn & 1, cy = (cn >> 1) & 1, cz = cn >> 2;
            const float w = (cx ? f[0] : 1.f - f[0]) * (cy ? f[1] : 1.f - f[1]) * (cz ? f[2] : 1.f - f[2]);
            const int t = ((l[2] + cz) * ey + (l[1] + cy)) * ex + (l[0] + cx);
            float v[8];
            tile_unpack<Gt>(sh.rec + t * W, v);
#pragma unroll
            for (int s = 0; s < 8; ++s) g[s] = fmaf(w, v[s], g[s]);
        }
    }
    __syncthreads();
    return true;
}

// D (q0 + dq) in position quanta, as a normalised float-float: D q0 with an exact
// product, D dq (|dq| << |q0|) folded into the low part.
__device__ __forceinline__ FF scale_q(FF D, float q0, float dq)
{
    const float p = __fmul_rn(D.hi, q0);
    float e = __fmaf_rn(D.hi, q0, -p);
    e = __fmaf_rn(D.lo, q0, e);
    e = __fmaf_rn(D.hi, dq, e);
    FF r;
    fast_two_sum(p, e, r.hi, r.lo);
    return r;
}

// SERIES: the drift correction as a power series (else a loop over the drift
// nodes); NK kick nodes are compile-time, so the loops unroll into constant-bank
// operands; UNI: every species has the same mass.
// TILE: the kicks gather from a shared-memory tile of the grid (tile_gather), with G's
// direct reads where a block's box is too large.
template <typename Gt, bool SERIES, int NK, bool UNI, bool TILE>
__global__ void __launch_bounds__(kThreads, 4) k_push_split(const __grid_constant__ PushArgs a,
                                                            uint32_t* __restrict__ X, const float* __restrict__ q0f,
                                                            float* __restrict__ dqf)
{
    __shared__ typename std::conditional<TILE, TileShared, int>::type tile_sh;
    const int64_t n = a.n;
    const uint32_t N = (uint32_t)a.N;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // block-uniform trip count (i0 is the same for every thread of a block)
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < n; i0 += stride) {
        const int64_t i = i0 + threadIdx.x;
        const bool live = i < n;
        SplitState cur{};
        if (live) cur = load_split(X, q0f, dqf, n, i);
        const int s = UNI || !live ? 0 : species_of(a, i);
        uint32_t X0 = cur.X0, X1 = cur.X1, X2 = cur.X2;
        const float qa = cur.qa, qb = cur.qb, qc = cur.qc;
        float da = cur.da, db = cur.db, dc = cur.dc;
        // |q0|^2 in float-float (exact squares), and |q0|^2 in FP32 for the kick
        const float pa = __fmul_rn(qa, qa), pb = __fmul_rn(qb, qb), pc = __fmul_rn(qc, qc);
        const float ea = __fmaf_rn(qa, qa, -pa), eb = __fmaf_rn(qb, qb, -pb), ec = __fmaf_rn(qc, qc, -pc);
        float s1, e1, s2, e2;
        two_sum(pa, pb, s1, e1);
        two_sum(s1, pc, s2, e2);
        const float elo = (e1 + e2) + (ea + eb + ec);
        const float q02 = s2;
        bool moved = false, kicked = false;
        for (int u = 0; u < a.nsub; ++u) {
            if (!TILE && !live) continue;
            const SubStep& st = a.sub[u];
            const SpeciesCoef& c = st.sp[s];
            if (live && st.do_drift) {
                // |q|^2 = |q0|^2 + (2 q0 + dq).dq; the second term is at most a few per
                // cent of the first and carries FP32 rounding only.
                const float small = fmaf(2.f * qa + da, da, fmaf(2.f * qb + db, db, (2.f * qc + dc) * dc));
                FF S;
                fast_two_sum(s2, elo + small, S.hi, S.lo);
                // D = sum_j Wd_j (S + mu_j)^-1/2 = r_c [sum_j Wd_j + sum_j Wd_j g(delta_j)],
                // r_c = (S + mu_c)^-1/2, delta_j = (mu_j - mu_c) r_c^2, g(d) = (1+d)^-1/2 - 1
                // = -d y / (1 + (1+d) y), y = (1+d)^-1/2.  The corrections are small next to
                // sum_j Wd_j, so hardware rsqrt and reciprocal (2^-22) suffice.  The weights
                // carry the factor 2^32/L, so D is in position quanta per eV.
                const FF r = ff_rsqrt(ff_add(S, c.mud_c));
                const float r2 = r.hi * r.hi;
                float corr = 0.f;
                if constexpr (SERIES) {
                    // g(delta_j) = sum_k c_k delta_j^k with delta_j = e_j t, so
                    // sum_j Wd_j g(delta_j) = sum_k Cd_k t^k (|e_j| <= 1/4, 0 <= t <= 1)
                    const float t = c.mud_c_f * r2;
                    corr = c.Cd[kTaylor - 1];
#pragma unroll
                    for (int k = kTaylor - 2; k >= 0; --k) corr = fmaf(corr, t, c.Cd[k]);
                    corr *= t;
                } else {
#pragma unroll
                    for (int j = 0; j < kMaxGL; ++j) {
                        if (j < a.n_gl) {
                            const float d = c.dmud_f[j] * r2;
                            const float t = 1.f + d;
                            const float y = rsqrtf(t);
                            corr = fmaf(c.Wd_f[j], -d * y * __frcp_rn(fmaf(t, y, 1.f)), corr);
                        }
                    }
                }
                FF A;
                fast_two_sum(c.Wd_sum.hi, __fadd_rn(c.Wd_sum.lo, corr), A.hi, A.lo);
                const FF D = ff_mul(r, A);
                X0 += round_mod32(scale_q(D, qa, da));
                X1 += round_mod32(scale_q(D, qb, db));
                X2 += round_mod32(scale_q(D, qc, dc));
                moved = true;
            }
            if (st.do_kick) {
                float g[8];
                bool tiled = false;
                if constexpr (TILE) tiled = tile_gather<Gt>(tile_sh, reinterpret_cast<const Gt*>(a.G[u]), N, live, X0,
                                                           X1, X2, g);
                if (!live) continue;
                if (!tiled) gather_order<Gt>(a.order, reinterpret_cast<const Gt*>(a.G[u]), N, X0, X1, X2, g);
                float Kpsi = 0.f, Kphi = 0.f;
#pragma unroll
                for (int j = 0; j < NK; ++j) {
                    const float e2k = q02 + c.muk_f[j];
                    const float ie = rsqrtf(e2k);
                    Kpsi = fmaf(c.Wk_f[j], e2k * ie, Kpsi);
                    Kphi = fmaf(c.Wk_f[j], ie, Kphi);
                }
                const float qdphi = qa * g[3] + qb * g[4] + qc * g[5];
                const float b = qdphi * Kphi + g[6] * c.dtau_k_f;
                const float a2 = q02 * Kphi;
                da += -g[0] * Kpsi - g[3] * a2 + qa * b;
                db += -g[1] * Kpsi - g[4] * a2 + qb * b;
                dc += -g[2] * Kpsi - g[5] * a2 + qc * b;
                kicked = true;
            }
        }
        if (live && kicked) {
            __stcs(dqf + i, da);
            __stcs(dqf + n + i, db);
            __stcs(dqf + 2 * n + i, dc);
        }
        if (live && moved) {
            __stcs(X + i, X0);
            __stcs(X + n + i, X1);
            __stcs(X + 2 * n + i, X2);
        }
    }
}

template <typename Gt, bool SERIES, bool UNI, bool TILE>
void push_split_tile(cudaStream_t s, unsigned b, const PushArgs& a, const ParticleState& st)
{
    switch (a.n_kick) {
        case 2: launch_pass(k_push_split<Gt, SERIES, 2, UNI, TILE>, b, s, a, st.X, st.q0f, st.dqf); break;
        case 3: launch_pass(k_push_split<Gt, SERIES, 3, UNI, TILE>, b, s, a, st.X, st.q0f, st.dqf); break;
        default: launch_pass(k_push_split<Gt, SERIES, 4, UNI, TILE>, b, s, a, st.X, st.q0f, st.dqf); break;
    }
}

template <typename Gt, bool SERIES, bool UNI>
void push_split_nk(cudaStream_t s, unsigned b, const PushArgs& a, const ParticleState& st)
{
    // the tile serves the trilinear read (order 1)
    if (a.tile_gather && a.order == 1) push_split_tile<Gt, SERIES, UNI, true>(s, b, a, st);
    else push_split_tile<Gt, SERIES, UNI, false>(s, b, a, st);
}

template <typename Gt, bool UNI>
void push_split(cudaStream_t s, unsigned b, const PushArgs& a, const ParticleState& st)
{
    if (a.drift_series) push_split_nk<Gt, true, UNI>(s, b, a, st);
    else push_split_nk<Gt, false, UNI>(s, b, a, st);
}

// ---- the fused leapfrog pass, FP64-state form --------------------------------------
// x and q are FP64 in HBM and in registers and are accumulated in FP64; q_0 is FP32.
// Every step integral is evaluated in FP64 (WideCoef):
//   drift  D = int dtau / sqrt(q^2 + m^2 a^2) = r gm(t),  r = (q^2 + m^2 a_c^2)^(-1/2),
//   kick   K_phi = int dtau / eps_0 = r0 gm(t0),  K_psi = int eps_0 dtau = (u0 r0) gp(t0),
// with the polynomial's leading terms in FP64 and the rest in FP32 (they add less
// than 1e-7 of the integral).  The kick, at most ~1e-3 of |q| per step, is formed in
// FP32 from the FP32 gradients and added to q in FP64.  GB300 runs FP64 arithmetic
// and FP64 <-> FP32 conversions at 1/64 of its FP32 rate, so every conversion goes
// through the integer pipe (d2f_bits, f2d_bits).

// p(t) = sum_k c_k t^k: the terms from k = NF64 up in FP32 (Horner, from tf, t in FP32),
// then the terms below NF64 in FP64
template <int NF64>
__device__ __forceinline__ double wide_poly(const WidePoly& P, double t, float tf)
{
    float tail = P.c32[kWideDeg - NF64];
#pragma unroll
    for (int k = kWideDeg - NF64 - 1; k >= 0; --k) tail = fmaf(tail, tf, P.c32[k]);
    double acc = f2d_bits(tail);
#pragma unroll
    for (int k = NF64 - 1; k >= 0; --k) acc = fma(acc, t, P.c64[k]);
    return acc;
}

// Periodic wrap into [0, L) (wrap_f64, a result equal to L mapping to 0), taken only
// when x left the box.  The test runs on the bit patterns (IEEE doubles order like
// integers when positive; a negative value has the sign bit), so only a warp with a
// wrapping particle spends FP64 instructions on it.
__device__ __forceinline__ double wrap_rare(double x, double L, double invL, long long Lbits)
{
    const long long b = __double_as_longlong(x);
    if (b >= Lbits || b < 0) x = wrap_f64(x, L, invL);
    return x;
}

// The step integrals of one sub-step.  The drift's D depends on |q|^2, the kick's K_phi
// and K_psi on |q0|^2 only: the two chains are independent of each other and of the
// gather, so the pass issues them back to back and the FP64 pipe overlaps their
// latencies and the gather's.
template <bool SERIES>
__device__ __forceinline__ double drift_integral(const SubStep& st, int s, int n_gl, const double q[3])
{
    if constexpr (SERIES) {
        if (!st.wide.massless[s]) {
            const double inv = st.wide.inv_muc[s];
            // v = 1 + |q|^2 / (m^2 a_c^2), t = 1/v, D = v^(-1/2) gm(t) / (m a_c)
            const double v = fma(fma(q[0], q[0], fma(q[1], q[1], q[2] * q[2])), inv, 1.0);
            const double rv = rsqrt_fp64(v);
            const double t = rv * rv;
            return rv * wide_poly<kWideD64>(st.wide.drift[s], t, d2f_bits(t));
        }
        return rsqrt_fp64(fma(q[0], q[0], fma(q[1], q[1], q[2] * q[2]))) * st.wide.wsum[s];
    } else {
        const double qq = fma(q[0], q[0], fma(q[1], q[1], q[2] * q[2]));
        const SpeciesCoef& sc = st.sp[s];
        double D = 0.0;
        for (int j = 0; j < n_gl; ++j) D = fma(sc.Wd[j], rsqrt_fp64(qq + sc.mud[j]), D);
        return D;
    }
}

template <bool SERIES>
__device__ __forceinline__ void kick_integrals(const SubStep& st, int s, int n_kick, double s0, float& Kpsif,
                                               float& Kphif)
{
    double Kpsi, Kphi;
    if constexpr (SERIES) {
        // needed to ~1e-9 (they scale a kick of at most ~1e-3 of |q|): r0 to first order,
        // t0 from FP32 (its error enters times the first coefficient, ~1e-3 of the integral)
        const double muk = st.wide.muk[s];
        const double u0 = s0 + muk;
        const double r0 = rsqrt_fp64_1(u0);
        const float r0f = d2f_bits(r0);
        const float t0f = d2f_bits(muk) * r0f * r0f;
        const double t0 = f2d_bits(t0f);
        Kphi = r0 * wide_poly<kWideK64>(st.wide.kphi, t0, t0f);
        Kpsi = (u0 * r0) * wide_poly<kWideK64>(st.wide.kpsi, t0, t0f);
    } else {
        const SpeciesCoef& sc = st.sp[s];
        Kpsi = 0.0;
        Kphi = 0.0;
        for (int j = 0; j < n_kick; ++j) {
            const double e2 = s0 + sc.muk[j];
            const double ie = rsqrt_fp64(e2);
            Kpsi = fma(sc.Wk[j], e2 * ie, Kpsi);
            Kphi = fma(sc.Wk[j], ie, Kphi);
        }
    }
    Kpsif = d2f_bits(Kpsi);
    Kphif = d2f_bits(Kphi);
}

// One particle through the sub-steps of a pass of the FP64-state form.
template <typename Gt, bool SERIES, bool UNI>
__device__ __forceinline__ void wide_particle(const PushArgs& a, double* __restrict__ xd, double* __restrict__ qd,
                                              const float* __restrict__ q0f, int64_t i)
{
    const int64_t n = a.n;
    const uint32_t N = (uint32_t)a.N;
    const float invh = (float)a.invh;
    const long long Lbits = __double_as_longlong(a.L);
    const int s = UNI ? 0 : species_of(a, i);
    double x[3] = {__ldcs(xd + i), __ldcs(xd + n + i), __ldcs(xd + 2 * n + i)};
    double q[3] = {__ldcs(qd + i), __ldcs(qd + n + i), __ldcs(qd + 2 * n + i)};
    const float qa = __ldcs(q0f + i), qb = __ldcs(q0f + n + i), qc = __ldcs(q0f + 2 * n + i);
    // |q0|^2: exact products of the FP32 components, summed in FP64 (once per pass)
    const double da = f2d_bits(qa), db = f2d_bits(qb), dc = f2d_bits(qc);
    const double s0 = fma(da, da, fma(db, db, dc * dc));
    const float q02 = d2f_bits(s0);
    bool moved = false, kicked = false;
    for (int u = 0; u < a.nsub; ++u) {
        const SubStep& st = a.sub[u];
        float Kpsif = 0.f, Kphif = 0.f;
        if (st.do_kick) kick_integrals<SERIES>(st, s, a.n_kick, s0, Kpsif, Kphif);
        if (st.do_drift) {
            const double D = drift_integral<SERIES>(st, s, a.n_gl, q);
#pragma unroll
            for (int d = 0; d < 3; ++d) x[d] = wrap_rare(fma(q[d], D, x[d]), a.L, a.invL, Lbits);
            moved = true;
        }
        if (st.do_kick) {
            float g[8];
            gather_wide<Gt>(a.order, reinterpret_cast<const Gt*>(a.G[u]), N, invh, x, g);
            const float qdphi = qa * g[3] + qb * g[4] + qc * g[5];
            const float b = qdphi * Kphif + g[6] * st.wide.dtau_k;
            const float a2 = q02 * Kphif;
            q[0] += f2d_bits(-g[0] * Kpsif - g[3] * a2 + qa * b);
            q[1] += f2d_bits(-g[1] * Kpsif - g[4] * a2 + qb * b);
            q[2] += f2d_bits(-g[2] * Kpsif - g[5] * a2 + qc * b);
            kicked = true;
        }
    }
    if (moved) {
        __stcs(xd + i, x[0]);
        __stcs(xd + n + i, x[1]);
        __stcs(xd + 2 * n + i, x[2]);
    }
    if (kicked) {
        __stcs(qd + i, q[0]);
        __stcs(qd + n + i, q[1]);
        __stcs(qd + 2 * n + i, q[2]);
    }
}

// P particles per thread in lockstep (i0 + 32 p, p < P; i0 < n): their chains are
// independent, so the FP64 pipe overlaps one particle's result latencies with the
// others' work.  A particle at or past n repeats particle i0's work and stores nothing.
template <typename Gt, bool SERIES, bool UNI, int P>
__device__ __forceinline__ void wide_particles(const PushArgs& a, double* __restrict__ xd, double* __restrict__ qd,
                                               const float* __restrict__ q0f, int64_t i0)
{
    const int64_t n = a.n;
    const uint32_t N = (uint32_t)a.N;
    const float invh = (float)a.invh;
    const long long Lbits = __double_as_longlong(a.L);
    int64_t idx[P];
    bool ok[P];
    int s[P];
    double x[P][3], q[P][3], s0[P];
    float q0[P][3], q02[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        idx[p] = i0 + 32 * p;
        ok[p] = idx[p] < n;
        if (!ok[p]) idx[p] = i0;
        const int64_t i = idx[p];
        s[p] = UNI ? 0 : species_of(a, i);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            x[p][d] = __ldcs(xd + d * n + i);
            q[p][d] = __ldcs(qd + d * n + i);
            q0[p][d] = __ldcs(q0f + d * n + i);
        }
        const double da = f2d_bits(q0[p][0]), db = f2d_bits(q0[p][1]), dc = f2d_bits(q0[p][2]);
        s0[p] = fma(da, da, fma(db, db, dc * dc));
        q02[p] = d2f_bits(s0[p]);
    }
    bool moved = false, kicked = false;
    for (int u = 0; u < a.nsub; ++u) {
        const SubStep& st = a.sub[u];
        float Kpsif[P], Kphif[P];
#pragma unroll
        for (int p = 0; p < P; ++p) {
            Kpsif[p] = 0.f;
            Kphif[p] = 0.f;
            if (st.do_kick) kick_integrals<SERIES>(st, s[p], a.n_kick, s0[p], Kpsif[p], Kphif[p]);
        }
        if (st.do_drift) {
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const double D = drift_integral<SERIES>(st, s[p], a.n_gl, q[p]);
#pragma unroll
                for (int d = 0; d < 3; ++d) x[p][d] = wrap_rare(fma(q[p][d], D, x[p][d]), a.L, a.invL, Lbits);
            }
            moved = true;
        }
        if (st.do_kick) {
#pragma unroll
            for (int p = 0; p < P; ++p) {
                float g[8];
                gather_wide<Gt>(a.order, reinterpret_cast<const Gt*>(a.G[u]), N, invh, x[p], g);
                const float qa = q0[p][0], qb = q0[p][1], qc = q0[p][2];
                const float qdphi = qa * g[3] + qb * g[4] + qc * g[5];
                const float b = qdphi * Kphif[p] + g[6] * st.wide.dtau_k;
                const float a2 = q02[p] * Kphif[p];
                q[p][0] += f2d_bits(-g[0] * Kpsif[p] - g[3] * a2 + qa * b);
                q[p][1] += f2d_bits(-g[1] * Kpsif[p] - g[4] * a2 + qb * b);
                q[p][2] += f2d_bits(-g[2] * Kpsif[p] - g[5] * a2 + qc * b);
            }
            kicked = true;
        }
    }
#pragma unroll
    for (int p = 0; p < P; ++p) {
        if (!ok[p]) continue;
        const int64_t i = idx[p];
        if (moved)
#pragma unroll
            for (int d = 0; d < 3; ++d) __stcs(xd + d * n + i, x[p][d]);
        if (kicked)
#pragma unroll
            for (int d = 0; d < 3; ++d) __stcs(qd + d * n + i, q[p][d]);
    }
}

// The pass kernel: P particles per thread, with three resident blocks per SM for P = 1
// (80 registers, 24 warps) and two for P = 2 (128 registers, 16 warps carrying 32
// particles each); the second shape measured faster (its pairs give the FP64 pipe two
// independent chains per thread to overlap).  Work is handed out at run time, 32 P
// consecutive particles to a warp at a time (a.ctr[0] counts the chunks taken; each
// warp claims its next chunk before working on the current one, so that the atomic's
// round trip overlaps the work): the pass ends together on every SM however its
// blocks were placed, and the particles in flight stay one stretch of the cell order,
// whose grid cells the gathers share in L2.  The last warp to finish (a.ctr[1] counts
// them) sets both counters back to zero for the next pass.

template <typename Gt, bool SERIES, bool UNI, int P>
__global__ void __launch_bounds__(kThreads, P == 2 ? 2 : 3) k_push_wide(const __grid_constant__ PushArgs a,
                                                                       double* __restrict__ xd,
                                                                       double* __restrict__ qd,
                                                                       const float* __restrict__ q0f)
{
    const unsigned lane = threadIdx.x & 31u;
    unsigned next = 0;   // chunk indices (n < 2^38)
    if (lane == 0) next = (unsigned)atomicAdd(a.ctr, 1ull);
    for (;;) {
        const unsigned c = __shfl_sync(0xffffffffu, next, 0);
        const int64_t i0 = (int64_t)c * (32 * P);
        if (i0 >= a.n) break;
        if (lane == 0) next = (unsigned)atomicAdd(a.ctr, 1ull);
        const int64_t i = i0 + lane;
        if (i < a.n) {
            if constexpr (P == 1) wide_particle<Gt, SERIES, UNI>(a, xd, qd, q0f, i);
            else wide_particles<Gt, SERIES, UNI, P>(a, xd, qd, q0f, i);
        }
    }
    if (lane == 0) {
        const unsigned long long warps = (unsigned long long)gridDim.x * (blockDim.x / 32);
        __threadfence();
        if (atomicAdd(a.ctr + 1, 1ull) == warps - 1) {
            a.ctr[0] = 0;
            a.ctr[1] = 0;
        }
    }
}

// The passes of several contexts in one launch (the request server): the particles of
// segment k are the global indices [seg[k].begin, seg[k].begin + args->n), each segment's
// pass arguments in device memory.  Every particle runs the arithmetic of k_push_wide.
template <typename Gt>
__global__ void __launch_bounds__(kThreads, 3) k_push_wide_multi(const __grid_constant__ MultiPass m)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g0 = (int64_t)blockIdx.x * blockDim.x; g0 < m.total; g0 += stride) {
        const int64_t g = g0 + threadIdx.x;
        if (g >= m.total) continue;
        int k = 0;
        while (k + 1 < m.nseg && g >= m.seg[k + 1].begin) ++k;
        const MultiPass::Seg& sg = m.seg[k];
        const PushArgs& a = *sg.args;
        if (a.wide_series) wide_particle<Gt, true, false>(a, sg.xd, sg.qd, sg.q0f, g - sg.begin);
        else wide_particle<Gt, false, false>(a, sg.xd, sg.qd, sg.q0f, g - sg.begin);
    }
}

template <typename Gt>
void push_wide(cudaStream_t s, unsigned b, const PushArgs& a, const ParticleState& st)
{
    // two particles per thread with the fitted integrals (the node loops keep one)
    if (a.pair && a.wide_series) {
        if (a.uniform_species) launch_pass(k_push_wide<Gt, true, true, 2>, b, s, a, st.xd, st.qd, st.q0f);
        else launch_pass(k_push_wide<Gt, true, false, 2>, b, s, a, st.xd, st.qd, st.q0f);
    } else if (a.wide_series) {
        if (a.uniform_species) launch_pass(k_push_wide<Gt, true, true, 1>, b, s, a, st.xd, st.qd, st.q0f);
        else launch_pass(k_push_wide<Gt, true, false, 1>, b, s, a, st.xd, st.qd, st.q0f);
    } else {
        if (a.uniform_species) launch_pass(k_push_wide<Gt, false, true, 1>, b, s, a, st.xd, st.qd, st.q0f);
        else launch_pass(k_push_wide<Gt, false, false, 1>, b, s, a, st.xd, st.qd, st.q0f);
    }
}

// ---- the fused leapfrog pass, plain FP64 form --------------------------------
// FDF_EOM_EXACT (eq:releq and eq:geodesic, not symplectic): each kick holds q at its
// own start in place of q0, and each drift is scaled by 1 + phi + psi, the slot 7 of
// the grid of the last kick read at the drift's starting point, carried in sd.
__global__ void __launch_bounds__(kThreads) k_push_f64(const __grid_constant__ PushArgs a, double* __restrict__ xd,
                                                       double* __restrict__ qd, const double* __restrict__ q0d,
                                                       double* __restrict__ sd)
{
    const int64_t n = a.n;
    const bool exact = a.eom == FDF_EOM_EXACT;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int s = (int)(i >= a.sp_begin[0]) + (int)(i >= a.sp_begin[1]) + (int)(i >= a.sp_begin[2]);
        double x[3] = {xd[i], xd[n + i], xd[2 * n + i]};
        double q[3] = {qd[i], qd[n + i], qd[2 * n + i]};
        const double q0[3] = {q0d[i], q0d[n + i], q0d[2 * n + i]};
        double metric = exact ? sd[i] : 0.0;      // phi + psi at the next drift's start
        bool moved = false, kicked = false;
        for (int u = 0; u < a.nsub; ++u) {
            const SubStep& st = a.sub[u];
            const SpeciesCoef& c = st.sp[s];
            if (st.do_drift) {
                const double qq = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
                double D = 0.0;
                for (int j = 0; j < a.n_gl; ++j) D += c.Wd[j] / sqrt(qq + c.mud[j]);
                if (exact) D *= 1.0 + metric;
#pragma unroll
                for (int d = 0; d < 3; ++d) x[d] = wrap_f64(x[d] + D * q[d], a.L, a.invL);
                moved = true;
            }
            if (st.do_kick) {
                double g[8];
                gather_f64_order(a.order, reinterpret_cast<const double*>(a.G[u]), a.N, a.invh, x, g);
                // the kick's momentum: q0 (the separable forms) or q at the kick's start
                const double qk[3] = {exact ? q[0] : q0[0], exact ? q[1] : q0[1], exact ? q[2] : q0[2]};
                const double q02 = qk[0] * qk[0] + qk[1] * qk[1] + qk[2] * qk[2];
                double Kpsi = 0.0, Kphi = 0.0;
                for (int j = 0; j < a.n_kick; ++j) {
                    const double e = sqrt(q02 + c.muk[j]);
                    Kpsi += c.Wk[j] * e;
                    Kphi += c.Wk[j] / e;
                }
                const double qdphi = qk[0] * g[3] + qk[1] * g[4] + qk[2] * g[5];
                // the terms of the kick by equation of motion (FDF_EOM_*): grad psi,
                // grad phi, q0 (q0.grad phi) and q0 phi_dot coefficients (FDF_EOM_EXACT
                // takes FDF_EOM_GEODESIC's with q in place of q0)
                double A = Kpsi, B = q02 * Kphi, C = Kphi, Dt = c.dtau_k;
                if (a.eom == FDF_EOM_CANONICAL) C = Dt = 0.0;
                else if (a.eom == FDF_EOM_SR_NEWTON) { A = Kpsi + q02 * Kphi; B = C = Dt = 0.0; }
                else if (a.eom == FDF_EOM_Q_SIMPLE) B = C = Dt = 0.0;
                else if (a.eom == FDF_EOM_NEWTONIAN) { A = c.Ka; B = C = Dt = 0.0; }
#pragma unroll
                for (int d = 0; d < 3; ++d)
                    q[d] += -g[d] * A - g[3 + d] * B + qk[d] * (qdphi * C) + qk[d] * (g[6] * Dt);
                if (exact) metric = g[7];
                kicked = true;
            }
        }
        if (exact && kicked) sd[i] = metric;
        if (moved) {
            xd[i] = x[0];
            xd[n + i] = x[1];
            xd[2 * n + i] = x[2];
        }
        if (kicked) {
            qd[i] = q[0];
            qd[n + i] = q[1];
            qd[2 * n + i] = q[2];
        }
    }
}

// ---- state read-back ------------------------------------------------------------
template <int F>
__device__ __forceinline__ void load_state(const ParticleState& st, int64_t n, int64_t i, double L, double x[3],
                                           double q[3])
{
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if constexpr (F != kFixed) {
            x[d] = st.xd[d * n + i];
            q[d] = st.qd[d * n + i];
        } else {
            x[d] = L * ((double)st.X[d * n + i] * 2.3283064365386963e-10);
            q[d] = (double)st.q0f[d * n + i] + (double)st.dqf[d * n + i];
        }
    }
}

template <int F>
__global__ void __launch_bounds__(kThreads) k_export(ParticleState st, int64_t n, int64_t begin, int64_t count,
                                                     double L, double T, double* __restrict__ xo,
                                                     double* __restrict__ qo, double* __restrict__ wo)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < count;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = begin + j;
        const int64_t o = (int64_t)st.id[i] - begin;
        double x[3], q[3];
        load_state<F>(st, n, i, L, x, q);
        if (xo) {
            xo[o] = x[0];
            xo[count + o] = x[1];
            xo[2 * count + o] = x[2];
        }
        if (qo) {
            qo[o] = q[0];
            qo[count + o] = q[1];
            qo[2 * count + o] = q[2];
        }
        if (wo) {
            if constexpr (F == kPlain) wo[o] = dfweight(norm3_rn(q), st.pmag[i], T);
            else wo[o] = (double)dfweight_split(norm3_rn(q), st.pmag[i], T);
        }
    }
}

// The pre-initial draw in particle-index order.  The FP32/BF16-grid forms' fixed-point
// positions and sampled momenta are the live state and follow the permutation (it
// sorts before the momentum transform); the plain form keeps them in id order.
// |q_sampled| follows the permutation in both forms.
template <int F>
__global__ void __launch_bounds__(kThreads) k_export_initial(ParticleState st, int64_t n, int64_t begin,
                                                             int64_t count, uint32_t* __restrict__ Xo,
                                                             double* __restrict__ po, double* __restrict__ qso)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < count;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = begin + j;
        const int64_t o = (int64_t)st.id[i] - begin;
        if (Xo) {
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if constexpr (F == kPlain) Xo[d * count + j] = st.X[d * n + i];
                else Xo[d * count + o] = st.X[d * n + i];
            }
        }
        if (po) po[o] = st.pmag[i];
        if (qso) {
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if constexpr (F == kPlain) qso[d * count + j] = st.qs[d * n + i];
                else qso[d * count + o] = st.qs[d * n + i];
            }
        }
    }
}

// ---- the four terms of eq:releq (Fig. 2) ------------------------------------------
// At each particle of [begin, begin + count), with the fields G of the current step:
// T1 = -eps grad psi, T2 = -(q^2/eps) grad phi, T3 = q (q.grad phi)/eps, T4 = q phi_dot,
// eps = sqrt(q^2 + m^2 a^2).  sums[0..3] accumulate |T_i|^2 and sums[4] |T1+T2+T3+T4|^2
// (FP64, one atomic addition per warp and quantity).
template <int F, typename Gt>
__global__ void __launch_bounds__(kThreads) k_accel_terms(ParticleState st, int64_t n, int64_t begin, int64_t count,
                                                          int64_t n_part, Masses ms, double a, int order, int N,
                                                          double L, const Gt* __restrict__ G,
                                                          double* __restrict__ sums)
{
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < count;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = begin + j;
        const double m = ms.m[i / n_part];
        double x[3], q[3], g[8];
        load_state<F>(st, n, i, L, x, q);
        if constexpr (F == kPlain) {
            gather_f64_order(order, reinterpret_cast<const double*>(G), N, (double)N / L, x, g);
        } else if constexpr (F == kWide) {
            float gf[8];
            gather_wide<Gt>(order, G, (uint32_t)N, (float)((double)N / L), x, gf);
#pragma unroll
            for (int s = 0; s < 8; ++s) g[s] = (double)gf[s];
        } else {
            float gf[8];
            gather_order<Gt>(order, G, (uint32_t)N, st.X[i], st.X[n + i], st.X[2 * n + i], gf);
#pragma unroll
            for (int s = 0; s < 8; ++s) g[s] = (double)gf[s];
        }
        const double qq = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
        const double eps = sqrt(qq + m * m * a * a);
        const double qdphi = q[0] * g[3] + q[1] * g[4] + q[2] * g[5];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double t1 = -eps * g[d], t2 = -(qq / eps) * g[3 + d], t3 = q[d] * qdphi / eps, t4 = q[d] * g[6];
            acc[0] += t1 * t1;
            acc[1] += t2 * t2;
            acc[2] += t3 * t3;
            acc[3] += t4 * t4;
            const double tot = t1 + t2 + t3 + t4;
            acc[4] += tot * tot;
        }
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        double v = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(sums + k, v);
    }
}

// The deposit's warp pre-sum: the lanes of `peers` (the lanes whose particles share a
// base cell, from __match_any_sync) add their values v[0..K) so that the lowest lane of
// the set holds the set's sums.  A pairwise tree over the set in lane order: at each
// level a lane at an even position within the remaining set adds the values of the next
// remaining lane above it, and the lanes at odd positions drop out; log2 of the set's
// size levels, every lane of the warp taking part in each (the ballot-and-shuffle
// segmented reduction of warp-aggregated atomics).
template <int K, typename T>
__device__ __forceinline__ void peer_sum(T (&v)[K], unsigned peers)
{
    const unsigned lane = threadIdx.x & 31u;
    unsigned above = peers & (0xfffffffeu << lane);   // the set's lanes above this one
    unsigned pos = __popc(peers & ((1u << lane) - 1u));   // this lane's position in the set
    while (__any_sync(0xffffffffu, above != 0u)) {
        const int src = above ? __ffs(above) - 1 : (int)lane;
        const bool take = above != 0u && !(pos & 1u);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const T t = __shfl_sync(0xffffffffu, v[k], src);
            if (take) v[k] += t;
        }
        above &= ~__ballot_sync(0xffffffffu, pos & 1u);
        pos >>= 1;
    }
}

template <int F, bool PRESUM>
__global__ void __launch_bounds__(kThreads) k_deposit(ParticleState st, int64_t n, int64_t begin, int64_t count,
                                                      int64_t n_part, Masses ms, double a, double T, int quantity,
                                                      int parity, int order, int N, double L,
                                                      double* __restrict__ grid)
{
    const double invh = (double)N / L;
    // Warp-uniform trips: the lanes of a warp take 32 consecutive particles (neighbours in
    // the bucket order of the last sort) and stay converged for the pre-sum.
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31u); j0 < count; j0 += stride) {
        const int64_t j = j0 + (threadIdx.x & 31u);
        bool live = j < count;
        const int64_t i = begin + (live ? j : 0);
        if (live && parity >= 0 && (int)(st.id[i] & 1u) != parity) live = false;
        if (!PRESUM && !live) continue;
        const double m = ms.m[i / n_part];
        double x[3], q[3];
        load_state<F>(st, n, i, L, x, q);
        const double qm = norm3_rn(q);
        double v = 1.0;
        if constexpr (F == kPlain) {
            const double eps = sqrt(qm * qm + m * m * a * a);
            if (quantity == FDF_Q_W_EPS) v = dfweight(qm, st.pmag[i], T) * eps;
            else if (quantity == FDF_Q_W) v = dfweight(qm, st.pmag[i], T);
            else if (quantity == FDF_Q_EPS) v = eps;
            else if (quantity >= FDF_Q_W_QX) v = dfweight(qm, st.pmag[i], T) * q[quantity - FDF_Q_W_QX];
        } else {
            // The FP32-grid forms deposit in FP32 arithmetic (FP64 sums): the weight's
            // argument p - |q| (a small difference) is formed in FP64 first, and the
            // kernel weights of an FP64 position take its fraction from FP64.
            const float qf = (float)qm;
            const float ma = (float)(m * a);
            const float eps = sqrtf(fmaf(qf, qf, ma * ma));
            const float w = dfweight_split(qm, st.pmag[i], T);
            if (quantity == FDF_Q_W_EPS) v = (double)(w * eps);
            else if (quantity == FDF_Q_W) v = (double)w;
            else if (quantity == FDF_Q_EPS) v = (double)eps;
            else if (quantity >= FDF_Q_W_QX) v = (double)(w * (float)q[quantity - FDF_Q_W_QX]);
        }
        // per axis: the kernel's nodes and weights (order 1: 2 nodes, order 2: 3), in the
        // form's deposit precision
        using Wt = typename std::conditional<F == kPlain, double, float>::type;
        int idx[3][3];
        Wt w[3][3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            double u;
            if constexpr (F != kFixed) {
                u = x[d] * invh;
            } else {
                const uint32_t Xd = st.X[d * n + i];
                u = (double)__umulhi(Xd, (uint32_t)N) + (double)(Xd * (uint32_t)N) * 2.3283064365386963e-10;
            }
            const double c = order == 2 ? floor(u + 0.5) : floor(u);
            const Wt e = (Wt)(u - c);
            int ii = (int)c;
            if (ii >= N) ii -= N;
            if (ii < 0) ii += N;
            if (order == 2) {
                idx[d][0] = ii == 0 ? N - 1 : ii - 1;
                idx[d][1] = ii;
                idx[d][2] = ii + 1 == N ? 0 : ii + 1;
                w[d][0] = Wt(0.5) * (Wt(0.5) - e) * (Wt(0.5) - e);
                w[d][1] = Wt(0.75) - e * e;
                w[d][2] = Wt(0.5) * (Wt(0.5) + e) * (Wt(0.5) + e);
            } else {
                idx[d][0] = ii;
                idx[d][1] = ii + 1 == N ? 0 : ii + 1;
                idx[d][2] = ii;
                w[d][0] = Wt(1) - e;
                w[d][1] = e;
                w[d][2] = Wt(0);
            }
        }
        const Wt vw = (Wt)v;
        if constexpr (PRESUM) {
            // Particles sharing the base cell share every node: one match on it, sums
            // over the set by shuffles, and one atomic per set and node.
            const unsigned key = live ? (unsigned)(((size_t)idx[2][0] * N + idx[1][0]) * N + idx[0][0]) : 0xffffffffu;
            const unsigned peers = __match_any_sync(0xffffffffu, key);
            const bool lead = live && (peers & ((1u << (threadIdx.x & 31u)) - 1u)) == 0u;
            if (order == 2) {
                double c[27];
#pragma unroll
                for (int k = 0; k < 27; ++k) c[k] = live ? (double)(w[0][k % 3] * w[1][(k / 3) % 3] * w[2][k / 9] * vw) : 0.0;
                peer_sum<27>(c, peers);
                if (lead) {
#pragma unroll
                    for (int k = 0; k < 27; ++k)
                        atomicAdd(grid + ((size_t)idx[2][k / 9] * N + idx[1][(k / 3) % 3]) * N + idx[0][k % 3], c[k]);
                }
            } else {
                double c[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) c[k] = live ? (double)(w[0][k & 1] * w[1][(k >> 1) & 1] * w[2][k >> 2] * vw) : 0.0;
                peer_sum<8>(c, peers);
                if (lead) {
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        atomicAdd(grid + ((size_t)idx[2][k >> 2] * N + idx[1][(k >> 1) & 1]) * N + idx[0][k & 1], c[k]);
                }
            }
        } else {
            const int m3 = order == 2 ? 3 : 2;
            for (int cz = 0; cz < m3; ++cz)
                for (int cy = 0; cy < m3; ++cy)
                    for (int cx = 0; cx < m3; ++cx) {
                        const Wt wt = w[0][cx] * w[1][cy] * w[2][cz];
                        const size_t cell = ((size_t)idx[2][cz] * N + idx[1][cy]) * N + idx[0][cx];
                        atomicAdd(grid + cell, (double)(wt * vw));
                    }
        }
    }
}

Masses masses_of(const double* m_ev)
{
    Masses ms;
    for (int s = 0; s < kMaxSpecies; ++s) ms.m[s] = m_ev[s];
    return ms;
}

}  // namespace

cudaError_t launch_initial(cudaStream_t s, int precision, const ParticleState& st, int64_t n, int64_t n_part,
                           const double* m_ev, double a0, double tau0, int order, int N, double L, const void* G)
{
    if (n <= 0) return cudaSuccess;
    const unsigned b = grid_for(n);
    const Masses ms = masses_of(m_ev);
    const int f = form_of(precision), gp = grid_prec(precision);
#define FDF_INITIAL(F_, Gt_) \
    k_initial<F_, Gt_><<<b, kThreads, 0, s>>>(st, n, n_part, ms, a0, tau0, order, N, L, (const Gt_*)G)
    if (f == kPlain) FDF_INITIAL(kPlain, double);
    else if (f == kWide && gp == FDF_PREC_F32) FDF_INITIAL(kWide, float);
    else if (f == kWide) FDF_INITIAL(kWide, __nv_bfloat16);
    else if (gp == FDF_PREC_F32) FDF_INITIAL(kFixed, float);
    else FDF_INITIAL(kFixed, __nv_bfloat16);
#undef FDF_INITIAL
    return cudaGetLastError();
}

cudaError_t launch_push(cudaStream_t s, int precision, const ParticleState& st, const PushArgs& a)
{
    if (a.n <= 0) return cudaSuccess;
    const int f = form_of(precision), gp = grid_prec(precision);
    if (f == kPlain) {
        launch_pass(k_push_f64, grid_for(a.n), s, a, st.xd, st.qd, st.q0d, st.sd);
    } else if (f == kWide) {
        // a persistent grid of pass_blocks resident blocks per SM, whose warps take chunks
        // of particles from the work counters
        if (!a.ctr) return cudaErrorInvalidValue;
        int64_t nb = (a.n + kThreads - 1) / kThreads;
        if (nb > a.grid_blocks) nb = a.grid_blocks;
        const unsigned b = (unsigned)(nb < 1 ? 1 : nb);
        if (gp == FDF_PREC_F32) push_wide<float>(s, b, a, st);
        else push_wide<__nv_bfloat16>(s, b, a, st);
    } else {
        const unsigned b = grid_for(a.n);
        if (gp == FDF_PREC_F32) {
            if (a.uniform_species) push_split<float, true>(s, b, a, st);
            else push_split<float, false>(s, b, a, st);
        } else {
            if (a.uniform_species) push_split<__nv_bfloat16, true>(s, b, a, st);
            else push_split<__nv_bfloat16, false>(s, b, a, st);
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_push_multi(cudaStream_t s, int grid_precision, const MultiPass& m, int grid_blocks)
{
    if (m.total <= 0) return cudaSuccess;
    int64_t nb = (m.total + kThreads - 1) / kThreads;
    if (nb > grid_blocks) nb = grid_blocks;
    const unsigned b = (unsigned)(nb < 1 ? 1 : nb);
    if (grid_precision == FDF_PREC_F32) launch_pass(k_push_wide_multi<float>, b, s, m);
    else launch_pass(k_push_wide_multi<__nv_bfloat16>, b, s, m);
    return cudaGetLastError();
}

cudaError_t launch_export(cudaStream_t s, int precision, const ParticleState& st, int64_t n, int64_t begin,
                          int64_t count, double L, double T_ev, double* x, double* q, double* w)
{
    if (count <= 0) return cudaSuccess;
    const unsigned b = grid_for(count);
    const int f = form_of(precision);
    if (f == kPlain) k_export<kPlain><<<b, kThreads, 0, s>>>(st, n, begin, count, L, T_ev, x, q, w);
    else if (f == kWide) k_export<kWide><<<b, kThreads, 0, s>>>(st, n, begin, count, L, T_ev, x, q, w);
    else k_export<kFixed><<<b, kThreads, 0, s>>>(st, n, begin, count, L, T_ev, x, q, w);
    return cudaGetLastError();
}

cudaError_t launch_export_initial(cudaStream_t s, int precision, const ParticleState& st, int64_t n, int64_t begin,
                                  int64_t count, uint32_t* X, double* p, double* qs)
{
    if (count <= 0) return cudaSuccess;
    const unsigned b = grid_for(count);
    // the FP64-state and split-state forms both sort before the transform
    if (form_of(precision) == kPlain)
        k_export_initial<kPlain><<<b, kThreads, 0, s>>>(st, n, begin, count, X, p, qs);
    else
        k_export_initial<kFixed><<<b, kThreads, 0, s>>>(st, n, begin, count, X, p, qs);
    return cudaGetLastError();
}

cudaError_t launch_accel_terms(cudaStream_t s, int precision, const ParticleState& st, int64_t n, int64_t begin,
                               int64_t count, int64_t n_part, const double* m_ev, double a, int order, int N,
                               double L, const void* G, double* sums)
{
    if (count <= 0) return cudaSuccess;
    const unsigned b = grid_for(count);
    const Masses ms = masses_of(m_ev);
    const int f = form_of(precision), gp = grid_prec(precision);
#define FDF_TERMS(F_, Gt_) \
    k_accel_terms<F_, Gt_><<<b, kThreads, 0, s>>>(st, n, begin, count, n_part, ms, a, order, N, L, (const Gt_*)G, sums)
    if (f == kPlain) FDF_TERMS(kPlain, double);
    else if (f == kWide && gp == FDF_PREC_F32) FDF_TERMS(kWide, float);
    else if (f == kWide) FDF_TERMS(kWide, __nv_bfloat16);
    else if (gp == FDF_PREC_F32) FDF_TERMS(kFixed, float);
    else FDF_TERMS(kFixed, __nv_bfloat16);
#undef FDF_TERMS
    return cudaGetLastError();
}

cudaError_t launch_deposit(cudaStream_t s, int precision, const ParticleState& st, int64_t n, int64_t begin,
                           int64_t count, int64_t n_part, const double* m_ev, double a, double T_ev, int quantity,
                           int parity, int order, int N, double L, bool presum, double* grid)
{
    if (count <= 0) return cudaSuccess;
    const unsigned b = grid_for(count);
    const Masses ms = masses_of(m_ev);
    const int f = form_of(precision);
#define FDF_DEPOSIT(F_, P_) \
    k_deposit<F_, P_><<<b, kThreads, 0, s>>>(st, n, begin, count, n_part, ms, a, T_ev, quantity, parity, order, N, L, \
                                             grid)
    if (f == kPlain && presum) FDF_DEPOSIT(kPlain, true);
    else if (f == kPlain) FDF_DEPOSIT(kPlain, false);
    else if (f == kWide && presum) FDF_DEPOSIT(kWide, true);
    else if (f == kWide) FDF_DEPOSIT(kWide, false);
    else if (presum) FDF_DEPOSIT(kFixed, true);
    else FDF_DEPOSIT(kFixed, false);
#undef FDF_DEPOSIT
    return cudaGetLastError();
}

}  // namespace fdf
