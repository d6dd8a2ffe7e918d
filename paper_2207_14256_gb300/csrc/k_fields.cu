// k_fields.cu -- potential-gradient grids at one scale factor (Sec. 2.1 of
// Elbers 2022: the potentials follow from the transfer functions by Fourier
// transform, and the grids are shared by all particles of a step).
//
// Eight real fields are built, packed in pairs into four complex transforms
// (a real field has a Hermitian spectrum, so F_a + i F_b transforms to
// f_a + i f_b):
//   P0 = d_x psi + i d_y psi     P1 = d_z psi + i d_x phi
//   P2 = d_y phi + i d_z phi     P3 = phi_dot + i psi
// (P3 = phi_dot + i (phi + psi) for the steps of the exact equations of motion, and
// phi_dot + i 0 for the steps of the separable forms, whose passes read no slot 7)
// with d_j f = sum_n i k_j T_f(k, a) R_n e^{i k.x}, phi_dot = a H dT_phi/dln a R.
// R_n is a Hermitian Gaussian field drawn from Philox4x32-10 addressed by the
// signed mode (so the realisation does not depend on the launch), with
// <|R_n|^2> = P_R(k)/V, P_R = 2 pi^2 A_s k^-3 (k/k_pivot)^(n_s-1).
//
// Three passes over the 4 x N^3 complex work arrays, each an inverse DFT of
// length N = N1 N2 along one axis (16 x 16 at N = 256): a line's N2 threads
// each hold N1 values in registers, transform them, twiddle, exchange through
// a padded transpose in shared memory and transform the other factor:
//   z: form the spectrum from the stored unit Gaussian field and the per-step
//      amplitude table, and transform along z;
//   y: transform along y;
//   x: transform along x and write the interleaved gather grid G[cell][8] as
//      whole 32-byte records.
#include <cuda_bf16.h>

#include <utility>

#include "device_math.cuh"

namespace fdf {

namespace {

// ---- in-register DFTs ----------------------------------------------------------
// e^{2 pi i j / 32}, j = 0..31 (exact zeros and ones on the axes).
#define C0 0.9807852804032304491262
#define C1 0.9238795325112867561282
#define C2 0.8314696123025452370788
#define C3 0.7071067811865475244008
#define C4 0.5555702330196022247428
#define C5 0.3826834323650897717285
#define C6 0.1950903220161282678483
__constant__ double2 kTw32d[32] = {
    {1, 0}, {C0, C6}, {C1, C5}, {C2, C4}, {C3, C3}, {C4, C2}, {C5, C1}, {C6, C0},
    {0, 1}, {-C6, C0}, {-C5, C1}, {-C4, C2}, {-C3, C3}, {-C2, C4}, {-C1, C5}, {-C0, C6},
    {-1, 0}, {-C0, -C6}, {-C1, -C5}, {-C2, -C4}, {-C3, -C3}, {-C4, -C2}, {-C5, -C1}, {-C6, -C0},
    {0, -1}, {C6, -C0}, {C5, -C1}, {C4, -C2}, {C3, -C3}, {C2, -C4}, {C1, -C5}, {C0, -C6}};
__constant__ float2 kTw32f[32] = {
    {1, 0}, {(float)C0, (float)C6}, {(float)C1, (float)C5}, {(float)C2, (float)C4}, {(float)C3, (float)C3},
    {(float)C4, (float)C2}, {(float)C5, (float)C1}, {(float)C6, (float)C0}, {0, 1}, {(float)-C6, (float)C0},
    {(float)-C5, (float)C1}, {(float)-C4, (float)C2}, {(float)-C3, (float)C3}, {(float)-C2, (float)C4},
    {(float)-C1, (float)C5}, {(float)-C0, (float)C6}, {-1, 0}, {(float)-C0, (float)-C6}, {(float)-C1, (float)-C5},
    {(float)-C2, (float)-C4}, {(float)-C3, (float)-C3}, {(float)-C4, (float)-C2}, {(float)-C5, (float)-C1},
    {(float)-C6, (float)-C0}, {0, -1}, {(float)C6, (float)-C0}, {(float)C5, (float)-C1}, {(float)C4, (float)-C2},
    {(float)C3, (float)-C3}, {(float)C2, (float)-C4}, {(float)C1, (float)-C5}, {(float)C0, (float)-C6}};
#undef C0
#undef C1
#undef C2
#undef C3
#undef C4
#undef C5
#undef C6

template <typename V> __device__ __forceinline__ V tw32(int j);
template <> __device__ __forceinline__ float2 tw32<float2>(int j) { return kTw32f[j]; }
template <> __device__ __forceinline__ double2 tw32<double2>(int j) { return kTw32d[j]; }

// Compile-time loops: f(Idx<I>) for I = 0..N-1, so that every register-array index
// below is a constant expression.
template <int I> struct Idx {
    __host__ __device__ constexpr operator int() const { return I; }
};
template <typename F, int... Is>
__device__ __forceinline__ void sfor_impl(F&& f, std::integer_sequence<int, Is...>)
{
    (f(Idx<Is>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void sfor(F&& f)
{
    sfor_impl(f, std::make_integer_sequence<int, N>{});
}

__host__ __device__ constexpr int bitrev(int i, int R)
{
    int j = 0;
    for (int b = 1; b < R; b <<= 1, i >>= 1) j = (j << 1) | (i & 1);
    return j;
}
__host__ __device__ constexpr int ilog2c(int R) { return R <= 1 ? 0 : 1 + ilog2c(R / 2); }

// In-place inverse DFT of R <= 32 values in registers, X_k = sum_n v_n e^{+2 pi i n k / R}:
// iterative radix-2 Cooley-Tukey on a bit-reversed copy.
template <int R, typename V>
__device__ __forceinline__ void dft_reg(V* v)
{
    sfor<R>([&](auto I) {
        constexpr int i = I, j = bitrev(I, R);
        if constexpr (i < j) {
            const V t = v[i];
            v[i] = v[j];
            v[j] = t;
        }
    });
    sfor<ilog2c(R)>([&](auto S) {
        constexpr int len = 2 << S;
        sfor<R / len>([&](auto B) {
            constexpr int i = B * len;
            sfor<len / 2>([&](auto K) {
                constexpr int k = K;
                const V u = v[i + k];
                V t = v[i + k + len / 2];
                if constexpr (k != 0) {
                    if constexpr (4 * k == len) t = cmuli(t);
                    else t = cmul(t, tw32<V>(k * (32 / len)));
                }
                v[i + k] = cadd(u, t);
                v[i + k + len / 2] = csub(u, t);
            });
        });
    });
}

// ---- the line transform: N = N1 N2, two levels ----------------------------------
// X[k1 + N1 k2] = sum_n2 w_N2^(n2 k2) [ w_N^(n2 k1) sum_n1 x[N2 n1 + n2] w_N1^(n1 k1) ],
// w_M = e^{2 pi i / M}.  Thread n2 holds x[N2 n1 + n2] (n1 = 0..N1-1), transforms them
// and applies w_N^(n2 k1); one padded shared-memory transpose; thread t then does
// the N2-point transforms of k1 = t, t + N2, ... (G = N1 / N2 of them).
template <int N> struct Split;
template <> struct Split<8> { static constexpr int N1 = 4, N2 = 2; };
template <> struct Split<16> { static constexpr int N1 = 4, N2 = 4; };
template <> struct Split<32> { static constexpr int N1 = 8, N2 = 4; };
template <> struct Split<64> { static constexpr int N1 = 8, N2 = 8; };
template <> struct Split<128> { static constexpr int N1 = 16, N2 = 8; };
template <> struct Split<256> { static constexpr int N1 = 16, N2 = 16; };
template <> struct Split<512> { static constexpr int N1 = 32, N2 = 16; };

template <int N> struct Shape {
    static constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2, G = N1 / N2;
    static constexpr int T = N2;                               // threads per line
    static constexpr int TS0 = N2 * (N1 + 1);                  // transpose buffer per line (elements)
    // y and z passes: TX lines (consecutive x) per block, lane = xo + TX t.
    static constexpr int TX0 = 128 / T > 16 ? 128 / T : 16;
    static constexpr int TX = TX0 < N ? TX0 : N;
    static constexpr int THREADS = TX * T;
    // Line stride of the y and z passes' transpose buffers, in elements of E bytes.  One
    // shared-memory wavefront serves 128 bytes: P = 128 / E consecutive lanes over P bank
    // groups.  Lane xo + TXl t touches element n2 (N1 + 1) + k of the line at xo * stride
    // (n2 = t, N1 + 1 odd).  With stride = P / TXl (mod P) for TXl < P (a wavefront spans
    // P / TXl values of t), else 1 (mod P), the P lanes fall in P distinct bank groups.
    template <int E, int TXl>
    __host__ __device__ static constexpr int line_stride()
    {
        constexpr int P = 128 / E;
        constexpr int S = TXl < P ? P / TXl : 1;
        return TS0 + ((S - TS0 % P) % P + P) % P;
    }
    // x pass: TL lines per block, lane = t + T lo; stride TSX = T (mod 16).
    static constexpr int TL0 = 128 / T;
    static constexpr int TL = TL0 < N ? TL0 : N;
    static constexpr int THREADS_X = TL * T;
    static constexpr int SX = T % 16;
    static constexpr int TSX = TS0 + ((SX - TS0 % 16) + 16) % 16;
    static constexpr int TWS = N2 * (N1 + 1);                  // per-thread twiddle rows, padded
    // z pass: 128 threads (its per-thread amplitudes live in shared memory).
    static constexpr int TZ0 = 128 / T;
    static constexpr int TZ = TZ0 < N ? TZ0 : N;
    static constexpr int THREADS_Z = TZ * T;
};

// Twiddles of the first level, w_N^(n2 k1) at [n2 (N1 + 1) + k1]: a thread reads its
// own row, and lanes with different n2 fall in different banks.
template <typename V, int N>
__device__ __forceinline__ void load_line_twiddles(V* s_tw2, const V* __restrict__ tw)
{
    constexpr int N1 = Shape<N>::N1, N2 = Shape<N>::N2;
    for (int i = threadIdx.x; i < N1 * N2; i += blockDim.x) {
        const int n2 = i / N1, k1 = i - n2 * N1;
        s_tw2[n2 * (N1 + 1) + k1] = tw[(n2 * k1) & (N - 1)];
    }
}

template <typename V, int N>
__device__ __forceinline__ void line_first(V* v, int n2, const V* __restrict__ s_tw, V* tr)
{
    constexpr int N1 = Shape<N>::N1;
    dft_reg<N1>(v);
    const V* row = s_tw + n2 * (N1 + 1);
    sfor<N1>([&](auto K1) { tr[n2 * (N1 + 1) + K1] = cmul(v[K1], row[K1]); });
}

// Second level for k1 = t + g N2; out(k2, value) receives X[k1 + N1 k2].
template <typename V, int N, typename Out>
__device__ __forceinline__ void line_second(int t, const V* tr, Out&& out)
{
    constexpr int N1 = Shape<N>::N1, N2 = Shape<N>::N2, G = Shape<N>::G;
    sfor<G>([&](auto Gi) {
        const int k1 = t + Gi * N2;
        V u[N2];
        sfor<N2>([&](auto N2i) { u[N2i] = tr[N2i * (N1 + 1) + k1]; });
        dft_reg<N2>(u);
        sfor<N2>([&](auto K2) { out(k1 + N1 * K2, u[K2]); });
    });
}

// ---- precision-dependent scalar math -------------------------------------
__device__ __forceinline__ float f_log(float x) { return logf(x); }
__device__ __forceinline__ double f_log(double x) { return log(x); }
__device__ __forceinline__ float f_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double f_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ void f_sincospi(float x, float* s, float* c) { sincospif(x, s, c); }
__device__ __forceinline__ void f_sincospi(double x, double* s, double* c) { sincospi(x, s, c); }

__device__ __forceinline__ int sidx(int j, int N) { return j < (N >> 1) ? j : j - N; }

// The unit Gaussian of mode (jx, jy, jz), R/sqrt(P_R/V): zero for the mean and the
// Nyquist planes, conj of the mirror mode for non-canonical n.  Drawn once per run
// by k_noise.
template <typename V>
__device__ __forceinline__ V mode_unit(const FieldArgs& a, int jx, int jy, int jz)
{
    using T = typename Real<V>::T;
    const int N = a.N;
    const int nx = sidx(jx, N), ny = sidx(jy, N), nz = sidx(jz, N);
    const int h = -(N >> 1);
    if (nx == h || ny == h || nz == h || (nx == 0 && ny == 0 && nz == 0)) return mk<V>(T(0), T(0));
    const bool canon = nz > 0 || (nz == 0 && (ny > 0 || (ny == 0 && nx > 0)));
    const int mx = canon ? nx : -nx, my = canon ? ny : -ny, mz = canon ? nz : -nz;
    const uint64_t pack = (uint64_t)(uint32_t)(mx + (1 << 20)) | ((uint64_t)(uint32_t)(my + (1 << 20)) << 21) |
                          ((uint64_t)(uint32_t)(mz + (1 << 20)) << 42);
    const uint4 w = philox4x32_10(make_uint4((uint32_t)pack, (uint32_t)(pack >> 32), 16u, 0u), a.key0, a.key1);
    const T u1 = (T)((w.x >> 8) + 1u) * (T)5.9604644775390625e-08;  // (0, 1]
    const T u2 = (T)(w.y >> 8) * (T)5.9604644775390625e-08;         // [0, 1)
    T s, c;
    f_sincospi((T)2 * u2, &s, &c);
    T re, im;
    if (a.fixed_amp) {
        re = c;
        im = s;
    } else {
        const T r = f_sqrt((T)-2 * f_log(u1)) * (T)0.70710678118654752440;
        re = r * c;
        im = r * s;
    }
    if (!canon) im = -im;
    return mk<V>(re, im);
}

template <typename V>
__global__ void __launch_bounds__(256) k_noise(FieldArgs a, V* __restrict__ R)
{
    const int N = a.N;
    const size_t N3 = (size_t)N * N * N;
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < N3; c += (size_t)gridDim.x * blockDim.x) {
        const int jx = (int)(c % N), jy = (int)((c / N) % N), jz = (int)(c / ((size_t)N * N));
        R[c] = mode_unit<V>(a, jx, jy, jz);
    }
}

// Packed spectrum p of a mode with unit Gaussian R and amplitudes (Apsi, Aphi, Adot):
//   P0 = i kx Apsi R + i (i ky Apsi R)      (d_x psi + i d_y psi)
//   P1 = i kz Apsi R + i (i kx Aphi R)      (d_z psi + i d_x phi)
//   P2 = i ky Aphi R + i (i kz Aphi R)      (d_y phi + i d_z phi)
//   P3 = Adot R + i Apsi R                  (phi_dot + i psi)
template <typename V>
__device__ __forceinline__ V packed(int p, V R, typename Real<V>::T Apsi, typename Real<V>::T Aphi,
                                    typename Real<V>::T Adot, typename Real<V>::T kx, typename Real<V>::T ky,
                                    typename Real<V>::T kz)
{
    const V iR = cmuli(R);
    switch (p) {
        case 0: return mk<V>(Apsi * (kx * iR.x - ky * R.x), Apsi * (kx * iR.y - ky * R.y));
        case 1: return mk<V>(kz * Apsi * iR.x - kx * Aphi * R.x, kz * Apsi * iR.y - kx * Aphi * R.y);
        case 2: return mk<V>(Aphi * (ky * iR.x - kz * R.x), Aphi * (ky * iR.y - kz * R.y));
        default: return mk<V>(Adot * R.x + Apsi * iR.x, Adot * R.y + Apsi * iR.y);
    }
}

// Per scale factor, in FP64, for every m = |n|^2 in [0, M): k = k_f sqrt(m),
// the amplitude sqrt(P_R(k)/V) = sqrt(2 pi^2 A_s / V) k^-3/2 (k/k_pivot)^((n_s-1)/2)
// times T_psi, T_phi and a H dT_phi/dln a, read bilinearly in (ln k, ln a) with
// clamping from the FP64 tables [3][na][nk].
template <typename T>
__global__ void __launch_bounds__(256) k_mode_table(FieldArgs a, int M, const double* __restrict__ tabs,
                                                    T* __restrict__ A)
{
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < M; m += gridDim.x * blockDim.x) {
        double v[3] = {0.0, 0.0, 0.0};
        if (m > 0) {
            const double k = a.kf * sqrt((double)m);
            const double lnk = log(k);
            const double amp = a.amp0 / (k * sqrt(k)) * exp(a.half_nsm1 * (lnk - a.lnkp));
            const double pos = (lnk - a.lnk0) * a.inv_dlnk;
            int ik;
            double fk;
            if (pos <= 0.0) {
                ik = 0;
                fk = 0.0;
            } else if (pos >= a.nk - 1) {
                ik = a.nk - 2;
                fk = 1.0;
            } else {
                ik = (int)pos;
                fk = pos - ik;
            }
            for (int t = 0; t < 3; ++t) {
                const double* r0 = tabs + ((size_t)t * a.na + a.ia) * a.nk;
                const double* r1 = r0 + a.nk;
                const double v0 = (1.0 - fk) * r0[ik] + fk * r0[ik + 1];
                const double v1 = (1.0 - fk) * r1[ik] + fk * r1[ik + 1];
                v[t] = amp * ((1.0 - a.fa) * v0 + a.fa * v1);
            }
            v[2] *= a.aH;
        }
        A[4 * m] = (T)v[0];
        A[4 * m + 1] = (T)v[1];
        A[4 * m + 2] = (T)v[2];
        A[4 * m + 3] = T(0);
    }
}

// One entry of the amplitude table (4 values per |n|^2, 16- or 32-byte aligned) in
// as few loads as the type allows.
__device__ __forceinline__ void amp_entry(const float* A, int m, float& ap, float& af, float& ad)
{
    const float4 v = __ldg(reinterpret_cast<const float4*>(A) + m);
    ap = v.x;
    af = v.y;
    ad = v.z;
}
__device__ __forceinline__ void amp_entry(const double* A, int m, double& ap, double& af, double& ad)
{
    const double2 u = __ldg(reinterpret_cast<const double2*>(A) + 2 * m);
    ap = u.x;
    af = u.y;
    ad = __ldg(A + 4 * m + 2);
}

// ---- pass z: spectrum + inverse DFT along z ---------------------------------
// Block (x-tile, jy): TX columns along z.  Each thread reads the unit Gaussians of
// its N1 modes once, with their amplitudes A[|n|^2] at this scale factor, then forms,
// transforms and writes each of the four packed grids in turn.
template <typename V, int N>
__global__ void __launch_bounds__(Shape<N>::THREADS_Z, sizeof(V) == 8 ? 4 : 2) k_fields_z(FieldArgs a,
                                                                  const typename Real<V>::T* __restrict__ A,
                                                                  const V* __restrict__ R, const V* __restrict__ tw,
                                                                  V* __restrict__ W0)
{
    using T = typename Real<V>::T;
    using S = Shape<N>;
    constexpr int TX = S::TZ, N1 = S::N1, N2 = S::N2, NT = S::THREADS_Z;
    constexpr int TSZ = S::template line_stride<sizeof(V), S::TZ>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* s_tw = reinterpret_cast<V*>(smem_raw);
    V* tr = s_tw + S::TWS;                                  // TX * TSZ
    T* As = reinterpret_cast<T*>(tr + TX * TSZ);            // [3][N1][NT]: each thread's own column
    load_line_twiddles<V, N>(s_tw, tw);
    const int xo = threadIdx.x % TX, t = threadIdx.x / TX;
    const int x0 = blockIdx.x * TX, jy = blockIdx.y;
    const int nx = sidx(x0 + xo, N), ny = sidx(jy, N), h = -(N >> 1);
    const T kf = (T)a.kf;
    const T kx = kf * (T)nx, ky = kf * (T)ny;
    const size_t NN = (size_t)N * N;
    V Rv[N1];
    sfor<N1>([&](auto I) { Rv[I] = R[(size_t)(N2 * I + t) * NN + (size_t)jy * N + x0 + xo]; });
    // The amplitudes depend on |n|^2 only, so the modes nz and -nz of a column share
    // them.  Mode z = N2 I + t mirrors to z' = N - z: for t > 0 that is thread N2 - t,
    // index N1 - 1 - I; for t = 0 it is thread 0, index (N1 - I) mod N1.  Each thread
    // looks up the first half of its modes (t = 0 also I = N1/2) and writes the
    // amplitudes into its own column and into its mirror partner's.
    {
        const int tp = t == 0 ? 0 : N2 - t;
        const int partner = xo + TX * tp;
        sfor<N1 / 2 + 1>([&](auto I) {
            if (I < N1 / 2 || t == 0) {
                const int z = N2 * I + t;
                const int nz = sidx(z, N);
                const int Ip = t == 0 ? (N1 - I) % N1 : N1 - 1 - I;
                T ap = T(0), af = T(0), ad = T(0);
                if (nx != h && ny != h && nz != h) amp_entry(A, nx * nx + ny * ny + nz * nz, ap, af, ad);
                As[(0 * N1 + I) * NT + threadIdx.x] = ap;
                As[(1 * N1 + I) * NT + threadIdx.x] = af;
                As[(2 * N1 + I) * NT + threadIdx.x] = ad;
                As[(0 * N1 + Ip) * NT + partner] = ap;
                As[(1 * N1 + Ip) * NT + partner] = af;
                As[(2 * N1 + Ip) * NT + partner] = ad;
            }
        });
    }
    __syncthreads();
    const size_t N3 = NN * N;
#pragma unroll 1
    for (int p = 0; p < 4; ++p) {
        // one branch per packed grid, so that each reads only the amplitudes it uses
        // (psi; psi and phi; phi; phi_dot and psi) from shared memory
        V v[N1];
        // Q = 4 is grid 3 with slot 7 = phi + psi (the exact drift's factor), Q = 5 grid 3
        // with slot 7 = 0 (phi_dot transformed alone)
        auto form = [&](auto Q) {
            constexpr int P = Q < 4 ? (int)Q : 3;
            sfor<N1>([&](auto I) {
                const T kz = kf * (T)sidx(N2 * I + t, N);
                const int o = I * NT + threadIdx.x;
                const T apsi = (P == 2 || Q == 5) ? T(0) : As[0 * N1 * NT + o];
                const T aphi = (P == 1 || P == 2 || Q == 4) ? As[1 * N1 * NT + o] : T(0);
                const T adot = (P == 3) ? As[2 * N1 * NT + o] : T(0);
                v[I] = packed<V>(P, Rv[I], Q == 4 ? apsi + aphi : apsi, aphi, adot, kx, ky, kz);
            });
        };
        switch (p) {
            case 0: form(Idx<0>{}); break;
            case 1: form(Idx<1>{}); break;
            case 2: form(Idx<2>{}); break;
            default:
                if (a.slot7 == kSlot7Sum) form(Idx<4>{});
                else if (a.slot7 == kSlot7Zero) form(Idx<5>{});
                else form(Idx<3>{});
                break;
        }
        line_first<V, N>(v, t, s_tw, tr + xo * TSZ);
        __syncthreads();
        V* dst = W0 + p * N3 + (size_t)jy * N + x0 + xo;
        line_second<V, N>(t, tr + xo * TSZ, [&](int z, V val) { dst[(size_t)z * NN] = val; });
        __syncthreads();
    }
}

// ---- pass y: inverse DFT along y --------------------------------------------
// Block (x-tile, jz, packed grid p): TX lines along y, read and written in rows of
// TX consecutive x.
template <typename V, int N>
__global__ void __launch_bounds__(Shape<N>::THREADS) k_fields_y(FieldArgs a, const V* __restrict__ tw,
                                                                const V* __restrict__ W0, V* __restrict__ W1)
{
    using S = Shape<N>;
    constexpr int TX = S::TX, N1 = S::N1, N2 = S::N2;
    constexpr int TS = S::template line_stride<sizeof(V), S::TX>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* s_tw = reinterpret_cast<V*>(smem_raw);
    V* tr = s_tw + S::TWS;
    load_line_twiddles<V, N>(s_tw, tw);
    const int xo = threadIdx.x % TX, t = threadIdx.x / TX;
    const int x0 = blockIdx.x * TX, jz = blockIdx.y, p = blockIdx.z;
    const size_t N3 = (size_t)N * N * N;
    const V* src = W0 + p * N3 + (size_t)jz * N * N + x0 + xo;
    V v[N1];
    sfor<N1>([&](auto N1i) { v[N1i] = src[(size_t)(N2 * N1i + t) * N]; });
    __syncthreads();
    line_first<V, N>(v, t, s_tw, tr + xo * TS);
    __syncthreads();
    V* dst = W1 + p * N3 + (size_t)jz * N * N + x0 + xo;
    line_second<V, N>(t, tr + xo * TS, [&](int y, V val) { dst[(size_t)y * N] = val; });
}

// ---- pass x: inverse DFT along x, interleave into G[cell][8] ----------------
// Block: TL consecutive x-lines (line index = jz * N + jy).  FP64 records go out in
// two halves: grid 0 is parked in shared memory and written with grid 1, grid 2
// with grid 3 (one parked grid instead of three doubles the resident blocks).  FP32
// and BF16 records go out in one piece: grids 0..2 are parked and written with grid 3.
template <typename Gt, typename V> struct GRec;
// FP64 records (64 bytes) are written in two halves (grids 0-1, then grids 2-3), each
// two whole 32-byte sectors; FP32 and BF16 records in one piece, which measured faster
// for them (FP32 halves: 232 -> 310 us per x pass at 256^3).
template <> struct GRec<float, float2> {
    static constexpr bool kHalves = false;
    // one 32-byte store per record (the record is 32-byte aligned)
    __device__ static void put(float* G, size_t cell, float2 a, float2 b, float2 c, float2 d)
    {
        float* g = G + 8 * cell;
        asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(g), "f"(a.x), "f"(a.y),
                     "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y), "f"(d.x), "f"(d.y)
                     : "memory");
    }
};
template <> struct GRec<double, double2> {
    static constexpr bool kHalves = true;
    __device__ static void put_half(double* G, size_t cell, int h, double2 a, double2 b)
    {
        double2* g = reinterpret_cast<double2*>(G) + 4 * cell + 2 * h;
        g[0] = a;
        g[1] = b;
    }
};
template <> struct GRec<__nv_bfloat16, float2> {
    static constexpr bool kHalves = false;
    __device__ static void put(__nv_bfloat16* G, size_t cell, float2 a, float2 b, float2 c, float2 d)
    {
        const __nv_bfloat162 h0 = __floats2bfloat162_rn(a.x, a.y), h1 = __floats2bfloat162_rn(b.x, b.y);
        const __nv_bfloat162 h2 = __floats2bfloat162_rn(c.x, c.y), h3 = __floats2bfloat162_rn(d.x, d.y);
        uint4 u;
        u.x = *reinterpret_cast<const uint32_t*>(&h0);
        u.y = *reinterpret_cast<const uint32_t*>(&h1);
        u.z = *reinterpret_cast<const uint32_t*>(&h2);
        u.w = *reinterpret_cast<const uint32_t*>(&h3);
        reinterpret_cast<uint4*>(G)[cell] = u;
    }
};

template <typename V, typename Gt, int N>
__global__ void __launch_bounds__(Shape<N>::THREADS_X) k_fields_x(FieldArgs a, const V* __restrict__ tw,
                                                                  const V* __restrict__ W1, Gt* __restrict__ G)
{
    using S = Shape<N>;
    using Rec = GRec<Gt, V>;
    constexpr int TL = S::TL, N1 = S::N1, N2 = S::N2, T = S::T, LS = N + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* s_tw = reinterpret_cast<V*>(smem_raw);
    V* tr = s_tw + S::TWS;          // TL * TSX
    V* park = tr + TL * S::TSX;     // TL * LS per parked grid (1 for halves, else 3)
    load_line_twiddles<V, N>(s_tw, tw);
    const int t = threadIdx.x % T, lo = threadIdx.x / T;
    const size_t N3 = (size_t)N * N * N;
    const size_t line = (size_t)blockIdx.x * TL + lo;
    // the next packed grid's line is loaded while this one is transformed
    V nxt[N1];
    sfor<N1>([&](auto N1i) { nxt[N1i] = W1[line * N + N2 * N1i + t]; });
#pragma unroll 1
    for (int p = 0; p < 4; ++p) {
        V v[N1];
        sfor<N1>([&](auto N1i) { v[N1i] = nxt[N1i]; });
        if (p < 3) {
            const V* src = W1 + (p + 1) * N3 + line * N;
            sfor<N1>([&](auto N1i) { nxt[N1i] = src[N2 * N1i + t]; });
        }
        __syncthreads();
        line_first<V, N>(v, t, s_tw, tr + lo * S::TSX);
        __syncthreads();
        if constexpr (Rec::kHalves) {
            // each thread parks and reads back only its own x values: no barrier needed
            V* pk = park + lo * LS;
            if ((p & 1) == 0) {
                line_second<V, N>(t, tr + lo * S::TSX, [&](int x, V val) { pk[x] = val; });
            } else {
                const int h = p >> 1;
                line_second<V, N>(t, tr + lo * S::TSX,
                                  [&](int x, V val) { Rec::put_half(G, line * N + x, h, pk[x], val); });
            }
        } else {
            if (p < 3) {
                V* pk = park + (p * TL + lo) * LS;
                line_second<V, N>(t, tr + lo * S::TSX, [&](int x, V val) { pk[x] = val; });
            } else {
                const V* p0 = park + lo * LS;
                const V* p1 = park + (TL + lo) * LS;
                const V* p2 = park + (2 * TL + lo) * LS;
                line_second<V, N>(t, tr + lo * S::TSX,
                                  [&](int x, V val) { Rec::put(G, line * N + x, p0[x], p1[x], p2[x], val); });
            }
        }
    }
}

// ---- conversions between G and [8][N^3] FP64 (test hooks) -------------------
template <typename Gt>
__device__ __forceinline__ double gval(const Gt* G, size_t cell, int s)
{
    if constexpr (sizeof(Gt) == 2) return (double)__bfloat162float(G[cell * 8 + s]);
    else return (double)G[cell * 8 + s];
}

template <typename Gt>
__global__ void k_fields_to_f64(size_t N3, const Gt* __restrict__ G, double* __restrict__ out, unsigned mask)
{
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < N3; c += (size_t)gridDim.x * blockDim.x)
        for (int s = 0; s < 8; ++s)
            if (mask & (1u << s)) out[s * N3 + c] = gval(G, c, s);
}

template <typename Gt>
__global__ void k_fields_from_f64(size_t N3, const double* __restrict__ in, Gt* __restrict__ G)
{
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < N3; c += (size_t)gridDim.x * blockDim.x)
        for (int s = 0; s < 8; ++s) {
            if constexpr (sizeof(Gt) == 2) G[c * 8 + s] = __float2bfloat16_rn((float)in[s * N3 + c]);
            else G[c * 8 + s] = (Gt)in[s * N3 + c];
        }
}

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes)
{
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename V, int N>
cudaError_t run_z(cudaStream_t s, const FieldArgs& a, const void* A, const void* R, const void* tw, void* W0)
{
    using S = Shape<N>;
    using T = typename Real<V>::T;
    constexpr int TSZ = S::template line_stride<sizeof(V), S::TZ>();
    const size_t sm = (size_t)(S::TWS + S::TZ * TSZ) * sizeof(V) + (size_t)3 * S::N1 * S::THREADS_Z * sizeof(T);
    cudaError_t e = set_smem(k_fields_z<V, N>, sm);
    if (e != cudaSuccess) return e;
    k_fields_z<V, N><<<dim3(N / S::TZ, N), S::THREADS_Z, sm, s>>>(a, (const T*)A, (const V*)R, (const V*)tw, (V*)W0);
    return cudaGetLastError();
}

template <typename V, int N>
cudaError_t run_y(cudaStream_t s, const FieldArgs& a, const void* tw, const void* W0, void* W1)
{
    using S = Shape<N>;
    constexpr int TS = S::template line_stride<sizeof(V), S::TX>();
    const size_t sm = (size_t)(S::TWS + S::TX * TS) * sizeof(V);
    cudaError_t e = set_smem(k_fields_y<V, N>, sm);
    if (e != cudaSuccess) return e;
    k_fields_y<V, N><<<dim3(N / S::TX, N, 4), S::THREADS, sm, s>>>(a, (const V*)tw, (const V*)W0, (V*)W1);
    return cudaGetLastError();
}

template <typename V, typename Gt, int N>
cudaError_t run_x(cudaStream_t s, const FieldArgs& a, const void* tw, const void* W1, void* G)
{
    using S = Shape<N>;
    const int parked = GRec<Gt, V>::kHalves ? 1 : 3;
    const size_t sm = (size_t)(S::TWS + S::TL * S::TSX + parked * S::TL * (N + 1)) * sizeof(V);
    cudaError_t e = set_smem(k_fields_x<V, Gt, N>, sm);
    if (e != cudaSuccess) return e;
    k_fields_x<V, Gt, N><<<(unsigned)((size_t)N * N / S::TL), S::THREADS_X, sm, s>>>(a, (const V*)tw, (const V*)W1,
                                                                                    (Gt*)G);
    return cudaGetLastError();
}

#define FDF_DISPATCH_N(N, CALL)                     \
    switch (N) {                                    \
        case 8: return CALL(8);                     \
        case 16: return CALL(16);                   \
        case 32: return CALL(32);                   \
        case 64: return CALL(64);                   \
        case 128: return CALL(128);                 \
        case 256: return CALL(256);                 \
        case 512: return CALL(512);                 \
        default: return cudaErrorInvalidValue;      \
    }

}  // namespace

// ---- super-steps: G = (1 - w) A + w B, element by element -------------------
__global__ void __launch_bounds__(256) k_interp_f32(size_t n4, const float4* __restrict__ A,
                                                    const float4* __restrict__ B, float w, float4* __restrict__ G)
{
    const float u = 1.f - w;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
        const float4 a = __ldcs(A + i), b = __ldcs(B + i);
        G[i] = make_float4(u * a.x + w * b.x, u * a.y + w * b.y, u * a.z + w * b.z, u * a.w + w * b.w);
    }
}

__global__ void __launch_bounds__(256) k_interp_f64(size_t n2, const double2* __restrict__ A,
                                                    const double2* __restrict__ B, double w,
                                                    double2* __restrict__ G)
{
    const double u = 1.0 - w;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n2; i += (size_t)gridDim.x * blockDim.x) {
        const double2 a = A[i], b = B[i];
        G[i] = make_double2(u * a.x + w * b.x, u * a.y + w * b.y);
    }
}

// BF16 cells (8 values, 16 bytes): interpolated in FP32, rounded to nearest
__global__ void __launch_bounds__(256) k_interp_bf16(size_t n, const uint4* __restrict__ A,
                                                     const uint4* __restrict__ B, float w, uint4* __restrict__ G)
{
    const float u = 1.f - w;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const uint4 a = A[i], b = B[i];
        const uint32_t ai[4] = {a.x, a.y, a.z, a.w}, bi[4] = {b.x, b.y, b.z, b.w};
        uint32_t o[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float lo = u * __uint_as_float(ai[k] << 16) + w * __uint_as_float(bi[k] << 16);
            const float hi = u * __uint_as_float(ai[k] & 0xFFFF0000u) + w * __uint_as_float(bi[k] & 0xFFFF0000u);
            const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
            o[k] = *reinterpret_cast<const uint32_t*>(&h);
        }
        G[i] = make_uint4(o[0], o[1], o[2], o[3]);
    }
}

int mode_table_size(int N) { return 3 * (N / 2 - 1) * (N / 2 - 1) + 1; }

cudaError_t launch_interp_grid(cudaStream_t s, int precision, int N, const void* A, const void* B, double w,
                               void* G)
{
    const size_t N3 = (size_t)N * N * N;
    const size_t items = precision == FDF_PREC_F64 ? 4 * N3 : (precision == FDF_PREC_F32 ? 2 * N3 : N3);
    size_t blocks = (items + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    if (precision == FDF_PREC_F64)
        k_interp_f64<<<(unsigned)blocks, 256, 0, s>>>(items, (const double2*)A, (const double2*)B, w, (double2*)G);
    else if (precision == FDF_PREC_F32)
        k_interp_f32<<<(unsigned)blocks, 256, 0, s>>>(items, (const float4*)A, (const float4*)B, (float)w,
                                                       (float4*)G);
    else
        k_interp_bf16<<<(unsigned)blocks, 256, 0, s>>>(items, (const uint4*)A, (const uint4*)B, (float)w, (uint4*)G);
    return cudaGetLastError();
}

cudaError_t launch_mode_table(cudaStream_t s, int precision, const FieldArgs& a, const double* tabs64, void* A)
{
    const int M = mode_table_size(a.N);
    const unsigned blocks = (unsigned)((M + 255) / 256);
    if (precision == FDF_PREC_F64) k_mode_table<double><<<blocks, 256, 0, s>>>(a, M, tabs64, (double*)A);
    else k_mode_table<float><<<blocks, 256, 0, s>>>(a, M, tabs64, (float*)A);
    return cudaGetLastError();
}

cudaError_t launch_noise(cudaStream_t s, int precision, const FieldArgs& a, void* R)
{
    const size_t N3 = (size_t)a.N * a.N * a.N;
    const unsigned blocks = (unsigned)((N3 + 255) / 256 < 152 * 32 ? (N3 + 255) / 256 : 152 * 32);
    if (precision == FDF_PREC_F64) k_noise<double2><<<blocks, 256, 0, s>>>(a, (double2*)R);
    else k_noise<float2><<<blocks, 256, 0, s>>>(a, (float2*)R);
    return cudaGetLastError();
}

cudaError_t launch_fields_z(cudaStream_t s, int precision, const FieldArgs& a, const void* A, const void* R,
                            const void* tw, void* W0)
{
#define Z64(n) run_z<double2, n>(s, a, A, R, tw, W0)
#define Z32(n) run_z<float2, n>(s, a, A, R, tw, W0)
    if (precision == FDF_PREC_F64) FDF_DISPATCH_N(a.N, Z64)
    FDF_DISPATCH_N(a.N, Z32)
#undef Z64
#undef Z32
}

cudaError_t launch_fields_y(cudaStream_t s, int precision, const FieldArgs& a, const void* tw, const void* W0,
                            void* W1)
{
#define Y64(n) run_y<double2, n>(s, a, tw, W0, W1)
#define Y32(n) run_y<float2, n>(s, a, tw, W0, W1)
    if (precision == FDF_PREC_F64) FDF_DISPATCH_N(a.N, Y64)
    FDF_DISPATCH_N(a.N, Y32)
#undef Y64
#undef Y32
}

cudaError_t launch_fields_x(cudaStream_t s, int precision, const FieldArgs& a, const void* tw, const void* W1,
                            void* G)
{
#define X64(n) run_x<double2, double, n>(s, a, tw, W1, G)
#define X32(n) run_x<float2, float, n>(s, a, tw, W1, G)
#define X16(n) run_x<float2, __nv_bfloat16, n>(s, a, tw, W1, G)
    if (precision == FDF_PREC_F64) FDF_DISPATCH_N(a.N, X64)
    if (precision == FDF_PREC_F32) FDF_DISPATCH_N(a.N, X32)
    FDF_DISPATCH_N(a.N, X16)
#undef X64
#undef X32
#undef X16
}

cudaError_t launch_fields_to_f64(cudaStream_t s, int precision, int N, const void* G, double* out, unsigned mask)
{
    const size_t N3 = (size_t)N * N * N;
    const unsigned blocks = (unsigned)((N3 + 255) / 256 < 152 * 32 ? (N3 + 255) / 256 : 152 * 32);
    if (precision == FDF_PREC_F64) k_fields_to_f64<double><<<blocks, 256, 0, s>>>(N3, (const double*)G, out, mask);
    else if (precision == FDF_PREC_F32)
        k_fields_to_f64<float><<<blocks, 256, 0, s>>>(N3, (const float*)G, out, mask);
    else k_fields_to_f64<__nv_bfloat16><<<blocks, 256, 0, s>>>(N3, (const __nv_bfloat16*)G, out, mask);
    return cudaGetLastError();
}

cudaError_t launch_fields_from_f64(cudaStream_t s, int precision, int N, const double* in, void* G)
{
    const size_t N3 = (size_t)N * N * N;
    const unsigned blocks = (unsigned)((N3 + 255) / 256 < 152 * 32 ? (N3 + 255) / 256 : 152 * 32);
    if (precision == FDF_PREC_F64) k_fields_from_f64<double><<<blocks, 256, 0, s>>>(N3, in, (double*)G);
    else if (precision == FDF_PREC_F32) k_fields_from_f64<float><<<blocks, 256, 0, s>>>(N3, in, (float*)G);
    else k_fields_from_f64<__nv_bfloat16><<<blocks, 256, 0, s>>>(N3, in, (__nv_bfloat16*)G);
    return cudaGetLastError();
}

}  // namespace fdf
