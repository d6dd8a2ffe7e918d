// k_fields.cu -- potential-gradient grids at one scale factor (Sec. 2.1 of
// Elbers 2022: the potentials follow from the transfer functions by Fourier
// transform, and the grids are shared by all particles of a step).
//
// Eight real fields are built, packed in pairs into four complex transforms
// (a real field has a Hermitian spectrum, so F_a + i F_b transforms to
// f_a + i f_b):
//   P0 = d_x psi + i d_y psi     P1 = d_z psi + i d_x phi
//   P2 = d_y phi + i d_z phi     P3 = phi_dot + i psi
// with d_j f = sum_n i k_j T_f(k, a) R_n e^{i k.x}, phi_dot = a H dT_phi/dln a R.
// R_n is a Hermitian Gaussian field drawn from Philox4x32-10 addressed by the
// signed mode (so the realisation does not depend on the launch), with
// <|R_n|^2> = P_R(k)/V, P_R = 2 pi^2 A_s k^-3 (k/k_pivot)^(n_s-1).
//
// Three passes over the 4 x N^3 complex work arrays, each an inverse DFT
// along one axis of tiles held in shared memory (Stockham autosort, radix 4
// and 2, an even number of stages so the result ends where it started):
//   z: generate the spectrum of a tile (no read) and transform along z;
//   y: transform along y;
//   x: transform along x and write the interleaved gather grid G[cell][8].
#include <cuda_bf16.h>

#include "device_math.cuh"

namespace fdf {

namespace {

constexpr int kThreads = 256;

template <typename V>
__device__ void smem_ifft_lines(V* a, V* b, int N, int logN, int nl, int ls, const V* __restrict__ tw)
{
    int n4 = logN >> 1, n2 = logN & 1;
    if ((n4 + n2) & 1) {
        n4 -= 1;
        n2 += 2;
    }
    int logNs = 0;
    V* src = a;
    V* dst = b;
    for (int st = 0; st < n2 + n4; ++st) {
        const int logR = st < n2 ? 1 : 2;
        const int lognb = logN - logR;
        const int nb = 1 << lognb;
        const int Ns = 1 << logNs;
        const int total = nl << lognb;
        const int twshift = logN - logNs - logR;
        for (int t = threadIdx.x; t < total; t += blockDim.x) {
            const int line = t >> lognb, j = t & (nb - 1);
            const int k = j & (Ns - 1);
            const V* in = src + line * ls;
            V* out = dst + line * ls;
            const int tws = k << twshift;
            if (logR == 1) {
                const V v0 = in[j];
                const V v1 = cmul(in[j + nb], tw[tws]);
                const int base = ((j >> logNs) << (logNs + 1)) + k;
                out[base] = cadd(v0, v1);
                out[base + Ns] = csub(v0, v1);
            } else {
                const V v0 = in[j];
                const V v1 = cmul(in[j + nb], tw[tws]);
                const V v2 = cmul(in[j + 2 * nb], tw[2 * tws]);
                const V v3 = cmul(in[j + 3 * nb], tw[3 * tws]);
                const V s02 = cadd(v0, v2), d02 = csub(v0, v2);
                const V s13 = cadd(v1, v3), d13 = cmuli(csub(v1, v3));
                const int base = ((j >> logNs) << (logNs + 2)) + k;
                out[base] = cadd(s02, s13);
                out[base + Ns] = cadd(d02, d13);
                out[base + 2 * Ns] = csub(s02, s13);
                out[base + 3 * Ns] = csub(d02, d13);
            }
        }
        __syncthreads();
        V* t = src;
        src = dst;
        dst = t;
        logNs += logR;
    }
}

// ---- precision-dependent scalar math -------------------------------------
__device__ __forceinline__ float f_log(float x) { return logf(x); }
__device__ __forceinline__ double f_log(double x) { return log(x); }
__device__ __forceinline__ float f_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double f_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ void f_sincospi(float x, float* s, float* c) { sincospif(x, s, c); }
__device__ __forceinline__ void f_sincospi(double x, double* s, double* c) { sincospi(x, s, c); }

__device__ __forceinline__ int sidx(int j, int N) { return j < (N >> 1) ? j : j - N; }

// The four packed spectra of one mode (jx, jy, jz).  A[m], m = |n|^2, holds the
// amplitude sqrt(P_R(k)/V) times T_psi, T_phi and a H dT_phi/dln a at this scale
// factor (built in FP64 by k_mode_table); the mode supplies its unit Gaussian.
template <typename V>
__device__ __forceinline__ void mode_values(const FieldArgs& a, const typename Real<V>::T* __restrict__ A, int jx,
                                            int jy, int jz, V out[4])
{
    using T = typename Real<V>::T;
    const int N = a.N;
    const int nx = sidx(jx, N), ny = sidx(jy, N), nz = sidx(jz, N);
    const int h = -(N >> 1);
    if (nx == h || ny == h || nz == h || (nx == 0 && ny == 0 && nz == 0)) {
        out[0] = out[1] = out[2] = out[3] = mk<V>(T(0), T(0));
        return;
    }
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
    const int m = nx * nx + ny * ny + nz * nz;
    const T Apsi = A[4 * m], Aphi = A[4 * m + 1], Adot = A[4 * m + 2];
    const T kf = (T)a.kf;
    const T kx = kf * (T)nx, ky = kf * (T)ny, kz = kf * (T)nz;
    const V R = mk<V>(re, im);
    const V iR = cmuli(R);
    // P0 = i kx Tpsi R + i (i ky Tpsi R) = Tpsi (kx iR - ky R)
    out[0] = mk<V>(Apsi * (kx * iR.x - ky * R.x), Apsi * (kx * iR.y - ky * R.y));
    // P1 = i kz Tpsi R - kx Tphi R
    out[1] = mk<V>(kz * Apsi * iR.x - kx * Aphi * R.x, kz * Apsi * iR.y - kx * Aphi * R.y);
    // P2 = i ky Tphi R - kz Tphi R
    out[2] = mk<V>(Aphi * (ky * iR.x - kz * R.x), Aphi * (ky * iR.y - kz * R.y));
    // P3 = aH dT R + i Tpsi R
    out[3] = mk<V>(Adot * R.x + Apsi * iR.x, Adot * R.y + Apsi * iR.y);
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

template <typename V>
__device__ void load_twiddles(V* s_tw, const V* __restrict__ tw, int N)
{
    for (int i = threadIdx.x; i < N; i += blockDim.x) s_tw[i] = tw[i];
}

// ---- pass z: spectrum + inverse DFT along z ---------------------------------
// Block (x-tile, jy): TX columns of N modes along z, all four packed spectra.
template <typename V, int TX>
__global__ void __launch_bounds__(kThreads) k_fields_z(FieldArgs a, const typename Real<V>::T* __restrict__ A,
                                                       const V* __restrict__ tw, V* __restrict__ W0)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = a.N, LS = N + 1;
    V* tiles = reinterpret_cast<V*>(smem_raw);
    V* scratch = tiles + 4 * TX * LS;
    V* s_tw = scratch + TX * LS;
    load_twiddles(s_tw, tw, N);
    const int x0 = blockIdx.x * TX, jy = blockIdx.y;
    for (int e = threadIdx.x; e < TX * N; e += blockDim.x) {
        const int xo = e % TX, z = e / TX;
        V v[4];
        mode_values<V>(a, A, x0 + xo, jy, z, v);
#pragma unroll
        for (int p = 0; p < 4; ++p) tiles[p * TX * LS + xo * LS + z] = v[p];
    }
    __syncthreads();
    for (int p = 0; p < 4; ++p) smem_ifft_lines(tiles + p * TX * LS, scratch, N, a.logN, TX, LS, s_tw);
    const size_t N3 = (size_t)N * N * N;
    for (int e = threadIdx.x; e < TX * N; e += blockDim.x) {
        const int xo = e % TX, z = e / TX;
        const size_t g = ((size_t)z * N + jy) * N + x0 + xo;
#pragma unroll
        for (int p = 0; p < 4; ++p) W0[p * N3 + g] = tiles[p * TX * LS + xo * LS + z];
    }
}

// ---- pass y: inverse DFT along y --------------------------------------------
// Block (x-tile, jz, packed grid p).
template <typename V, int TX>
__global__ void __launch_bounds__(kThreads) k_fields_y(FieldArgs a, const V* __restrict__ tw,
                                                       const V* __restrict__ W0, V* __restrict__ W1)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = a.N, LS = N + 1;
    V* tile = reinterpret_cast<V*>(smem_raw);
    V* scratch = tile + TX * LS;
    V* s_tw = scratch + TX * LS;
    load_twiddles(s_tw, tw, N);
    const int x0 = blockIdx.x * TX, jz = blockIdx.y, p = blockIdx.z;
    const size_t N3 = (size_t)N * N * N;
    const V* src = W0 + p * N3 + (size_t)jz * N * N + x0;
    for (int e = threadIdx.x; e < TX * N; e += blockDim.x) {
        const int xo = e % TX, y = e / TX;
        tile[xo * LS + y] = src[(size_t)y * N + xo];
    }
    __syncthreads();
    smem_ifft_lines(tile, scratch, N, a.logN, TX, LS, s_tw);
    V* dst = W1 + p * N3 + (size_t)jz * N * N + x0;
    for (int e = threadIdx.x; e < TX * N; e += blockDim.x) {
        const int xo = e % TX, y = e / TX;
        dst[(size_t)y * N + xo] = tile[xo * LS + y];
    }
}

// ---- pass x: inverse DFT along x, interleave into G[cell][8] ----------------
template <typename G> struct GStore;
template <> struct GStore<float> {
    __device__ static void put(float* G, size_t cell, const float v[8])
    {
        float4* g = reinterpret_cast<float4*>(G) + 2 * cell;
        g[0] = make_float4(v[0], v[1], v[2], v[3]);
        g[1] = make_float4(v[4], v[5], v[6], v[7]);
    }
};
template <> struct GStore<double> {
    __device__ static void put(double* G, size_t cell, const double v[8])
    {
        double2* g = reinterpret_cast<double2*>(G) + 4 * cell;
        g[0] = make_double2(v[0], v[1]);
        g[1] = make_double2(v[2], v[3]);
        g[2] = make_double2(v[4], v[5]);
        g[3] = make_double2(v[6], v[7]);
    }
};
template <> struct GStore<__nv_bfloat16> {
    __device__ static void put(__nv_bfloat16* G, size_t cell, const float v[8])
    {
        uint4 u;
        __nv_bfloat162 h0 = __floats2bfloat162_rn(v[0], v[1]);
        __nv_bfloat162 h1 = __floats2bfloat162_rn(v[2], v[3]);
        __nv_bfloat162 h2 = __floats2bfloat162_rn(v[4], v[5]);
        __nv_bfloat162 h3 = __floats2bfloat162_rn(v[6], v[7]);
        u.x = *reinterpret_cast<uint32_t*>(&h0);
        u.y = *reinterpret_cast<uint32_t*>(&h1);
        u.z = *reinterpret_cast<uint32_t*>(&h2);
        u.w = *reinterpret_cast<uint32_t*>(&h3);
        reinterpret_cast<uint4*>(G)[cell] = u;
    }
};

// Block: TL consecutive x-lines (line index = jz * N + jy), all four grids.
template <typename V, typename Gt, int TL>
__global__ void __launch_bounds__(kThreads) k_fields_x(FieldArgs a, const V* __restrict__ tw,
                                                       const V* __restrict__ W1, Gt* __restrict__ G)
{
    using T = typename Real<V>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = a.N, LS = N + 1;
    V* tiles = reinterpret_cast<V*>(smem_raw);
    V* scratch = tiles + 4 * TL * LS;
    V* s_tw = scratch + TL * LS;
    load_twiddles(s_tw, tw, N);
    const size_t N3 = (size_t)N * N * N;
    const size_t l0 = (size_t)blockIdx.x * TL;
    for (int e = threadIdx.x; e < TL * N; e += blockDim.x) {
        const int lo = e / N, x = e - lo * N;
#pragma unroll
        for (int p = 0; p < 4; ++p) tiles[p * TL * LS + lo * LS + x] = W1[p * N3 + (l0 + lo) * N + x];
    }
    __syncthreads();
    for (int p = 0; p < 4; ++p) smem_ifft_lines(tiles + p * TL * LS, scratch, N, a.logN, TL, LS, s_tw);
    for (int e = threadIdx.x; e < TL * N; e += blockDim.x) {
        const int lo = e / N, x = e - lo * N;
        T v[8];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const V c = tiles[p * TL * LS + lo * LS + x];
            v[2 * p] = c.x;
            v[2 * p + 1] = c.y;
        }
        if constexpr (sizeof(Gt) == 2) {
            float f[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) f[i] = (float)v[i];
            GStore<Gt>::put(G, (l0 + lo) * N + x, f);
        } else {
            GStore<Gt>::put(G, (l0 + lo) * N + x, v);
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
__global__ void k_fields_to_f64(size_t N3, const Gt* __restrict__ G, double* __restrict__ out)
{
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < N3; c += (size_t)gridDim.x * blockDim.x)
        for (int s = 0; s < 8; ++s) out[s * N3 + c] = gval(G, c, s);
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

constexpr int kTile = 8;

template <typename V>
size_t smem_z(int N)
{
    return (size_t)(5 * kTile * (N + 1) + N) * sizeof(V);
}
template <typename V>
size_t smem_y(int N)
{
    return (size_t)(2 * kTile * (N + 1) + N) * sizeof(V);
}
template <typename V>
size_t smem_x(int N)
{
    return (size_t)(5 * kTile * (N + 1) + N) * sizeof(V);
}

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes)
{
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

int mode_table_size(int N) { return 3 * (N / 2 - 1) * (N / 2 - 1) + 1; }

cudaError_t launch_mode_table(cudaStream_t s, int precision, const FieldArgs& a, const double* tabs64, void* A)
{
    const int M = mode_table_size(a.N);
    const unsigned blocks = (unsigned)((M + 255) / 256);
    if (precision == FDF_PREC_F64) k_mode_table<double><<<blocks, 256, 0, s>>>(a, M, tabs64, (double*)A);
    else k_mode_table<float><<<blocks, 256, 0, s>>>(a, M, tabs64, (float*)A);
    return cudaGetLastError();
}

cudaError_t launch_fields_z(cudaStream_t s, int precision, const FieldArgs& a, const void* A, const void* tw,
                            void* W0)
{
    const dim3 grid(a.N / kTile, a.N);
    if (precision == FDF_PREC_F64) {
        const size_t sm = smem_z<double2>(a.N);
        cudaError_t e = set_smem(k_fields_z<double2, kTile>, sm);
        if (e != cudaSuccess) return e;
        k_fields_z<double2, kTile><<<grid, kThreads, sm, s>>>(a, (const double*)A, (const double2*)tw,
                                                              (double2*)W0);
    } else {
        const size_t sm = smem_z<float2>(a.N);
        cudaError_t e = set_smem(k_fields_z<float2, kTile>, sm);
        if (e != cudaSuccess) return e;
        k_fields_z<float2, kTile><<<grid, kThreads, sm, s>>>(a, (const float*)A, (const float2*)tw, (float2*)W0);
    }
    return cudaGetLastError();
}

cudaError_t launch_fields_y(cudaStream_t s, int precision, const FieldArgs& a, const void* tw, const void* W0,
                            void* W1)
{
    const dim3 grid(a.N / kTile, a.N, 4);
    if (precision == FDF_PREC_F64) {
        const size_t sm = smem_y<double2>(a.N);
        cudaError_t e = set_smem(k_fields_y<double2, kTile>, sm);
        if (e != cudaSuccess) return e;
        k_fields_y<double2, kTile><<<grid, kThreads, sm, s>>>(a, (const double2*)tw, (const double2*)W0,
                                                              (double2*)W1);
    } else {
        const size_t sm = smem_y<float2>(a.N);
        cudaError_t e = set_smem(k_fields_y<float2, kTile>, sm);
        if (e != cudaSuccess) return e;
        k_fields_y<float2, kTile><<<grid, kThreads, sm, s>>>(a, (const float2*)tw, (const float2*)W0, (float2*)W1);
    }
    return cudaGetLastError();
}

cudaError_t launch_fields_x(cudaStream_t s, int precision, const FieldArgs& a, const void* tw, const void* W1,
                            void* G)
{
    const unsigned blocks = (unsigned)((size_t)a.N * a.N / kTile);
    if (precision == FDF_PREC_F64) {
        const size_t sm = smem_x<double2>(a.N);
        cudaError_t e = set_smem(k_fields_x<double2, double, kTile>, sm);
        if (e != cudaSuccess) return e;
        k_fields_x<double2, double, kTile><<<blocks, kThreads, sm, s>>>(a, (const double2*)tw, (const double2*)W1,
                                                                       (double*)G);
    } else if (precision == FDF_PREC_F32) {
        const size_t sm = smem_x<float2>(a.N);
        cudaError_t e = set_smem(k_fields_x<float2, float, kTile>, sm);
        if (e != cudaSuccess) return e;
        k_fields_x<float2, float, kTile><<<blocks, kThreads, sm, s>>>(a, (const float2*)tw, (const float2*)W1,
                                                                     (float*)G);
    } else {
        const size_t sm = smem_x<float2>(a.N);
        cudaError_t e = set_smem(k_fields_x<float2, __nv_bfloat16, kTile>, sm);
        if (e != cudaSuccess) return e;
        k_fields_x<float2, __nv_bfloat16, kTile><<<blocks, kThreads, sm, s>>>(a, (const float2*)tw,
                                                                             (const float2*)W1, (__nv_bfloat16*)G);
    }
    return cudaGetLastError();
}

cudaError_t launch_fields_to_f64(cudaStream_t s, int precision, int N, const void* G, double* out)
{
    const size_t N3 = (size_t)N * N * N;
    const unsigned blocks = (unsigned)((N3 + 255) / 256 < 152 * 32 ? (N3 + 255) / 256 : 152 * 32);
    if (precision == FDF_PREC_F64) k_fields_to_f64<double><<<blocks, 256, 0, s>>>(N3, (const double*)G, out);
    else if (precision == FDF_PREC_F32) k_fields_to_f64<float><<<blocks, 256, 0, s>>>(N3, (const float*)G, out);
    else k_fields_to_f64<__nv_bfloat16><<<blocks, 256, 0, s>>>(N3, (const __nv_bfloat16*)G, out);
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
