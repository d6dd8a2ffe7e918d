// k_sort.cu -- re-bucketing of particles by position for gather locality.
//
// Each particle's arithmetic is independent of the others (the metric is
// computed beforehand in linear theory, Sec. 2.1), so the particle arrays may
// be permuted freely; results are read back by particle id.  Particles are
// ordered by key = species * B + Morton(tile), the tile being a cube of
// ts^3 cells (B tiles per species), with a counting sort:
//   keys:    key of every particle and a histogram of keys;
//   scan:    exclusive prefix sum of the histogram (three small passes);
//   scatter: every particle's state moves to offset[key]++ in the other half
//            of the double-buffered state.
// Within a tile the order is whatever the atomics produce; no result depends
// on it.
#include "device_math.cuh"

namespace fdf {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ uint32_t spread3(uint32_t v)  // 10 bits -> every third bit
{
    v &= 0x3FFu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

template <int Prec>
__global__ void __launch_bounds__(kThreads) k_sort_keys(ParticleState st, int64_t n, int64_t n_part, uint32_t N,
                                                        int tile_shift, uint32_t tiles_per_species, double invh,
                                                        uint32_t* __restrict__ key, uint32_t* __restrict__ hist)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t c[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if constexpr (Prec == FDF_PREC_F64) {
                int ci = (int)floor(st.xd[d * n + i] * invh);
                ci = ci < 0 ? 0 : (ci >= (int)N ? (int)N - 1 : ci);
                c[d] = (uint32_t)ci;
            } else {
                c[d] = __umulhi(st.X[d * n + i], N);
            }
            c[d] >>= tile_shift;
        }
        const uint32_t s = (uint32_t)(i / n_part);
        const uint32_t k = s * tiles_per_species + (spread3(c[0]) | (spread3(c[1]) << 1) | (spread3(c[2]) << 2));
        key[i] = k;
        atomicAdd(hist + k, 1u);
    }
}

// Exclusive scan, phase 1: each block scans 4 * kThreads elements.
__global__ void __launch_bounds__(kThreads) k_scan_local(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                                         uint32_t* __restrict__ bsum, int n)
{
    __shared__ uint32_t warp_tot[kThreads / 32];
    const int base = blockIdx.x * 4 * kThreads + 4 * threadIdx.x;
    uint32_t v[4], t = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        v[j] = base + j < n ? in[base + j] : 0u;
        t += v[j];
    }
    // inclusive scan of the thread totals within the block
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t x = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = lane < kThreads / 32 ? warp_tot[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kThreads / 32) warp_tot[lane] = w;
    }
    __syncthreads();
    uint32_t run = x - t + (wid ? warp_tot[wid - 1] : 0u);  // exclusive prefix of this thread
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (base + j < n) out[base + j] = run;
        run += v[j];
    }
    if (threadIdx.x == kThreads - 1) bsum[blockIdx.x] = run;
}

// Phase 2: one block scans the block totals (at most 4 * kThreads of them).
__global__ void __launch_bounds__(kThreads) k_scan_totals(uint32_t* __restrict__ bsum, int nb)
{
    __shared__ uint32_t s[4 * kThreads];
    for (int i = threadIdx.x; i < 4 * kThreads; i += kThreads) s[i] = i < nb ? bsum[i] : 0u;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int i = 0; i < nb; ++i) {
            const uint32_t v = s[i];
            s[i] = run;
            run += v;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += kThreads) bsum[i] = s[i];
}

// Phase 3: add the block offsets.
__global__ void __launch_bounds__(kThreads) k_scan_add(uint32_t* __restrict__ out, const uint32_t* __restrict__ bsum,
                                                       int n)
{
    const int base = blockIdx.x * 4 * kThreads;
    const uint32_t add = bsum[blockIdx.x];
    for (int j = threadIdx.x; j < 4 * kThreads; j += kThreads)
        if (base + j < n) out[base + j] += add;
}

template <int Prec>
__global__ void __launch_bounds__(kThreads) k_sort_scatter(ParticleState a, ParticleState b, int64_t n,
                                                           const uint32_t* __restrict__ key,
                                                           uint32_t* __restrict__ offset)
{
    // Grid-stride loop with a warp-uniform trip count, so that every lane can take
    // part in the warp-aggregated atomic: lanes sharing a key (the common case once
    // the state is nearly sorted) take one atomicAdd through their leader.
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x; i0 < n; i0 += stride) {
        const int64_t i = i0 + threadIdx.x;
        const bool live = i < n;
        const unsigned active = __ballot_sync(0xffffffffu, live);
        if (!live) continue;
        const uint32_t k = key[i];
        const unsigned peers = __match_any_sync(active, k);
        const int lane = threadIdx.x & 31;
        const int leader = __ffs(peers) - 1;
        const unsigned rank = __popc(peers & ((1u << lane) - 1u));
        uint32_t base = 0;
        if (lane == leader) base = atomicAdd(offset + k, (uint32_t)__popc(peers));
        base = __shfl_sync(peers, base, leader);
        const int64_t j = (int64_t)base + rank;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if constexpr (Prec == FDF_PREC_F64) {
                b.xd[d * n + j] = a.xd[d * n + i];
                b.qd[d * n + j] = a.qd[d * n + i];
                b.q0d[d * n + j] = a.q0d[d * n + i];
            } else {
                b.X[d * n + j] = a.X[d * n + i];
                b.q0f[d * n + j] = a.q0f[d * n + i];
                b.dqf[d * n + j] = a.dqf[d * n + i];
            }
        }
        b.pmag[j] = a.pmag[i];
        b.id[j] = a.id[i];
    }
}

unsigned grid_for(int64_t n)
{
    int64_t b = (n + kThreads - 1) / kThreads;
    if (b > 152 * 16) b = 152 * 16;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

int sort_tile_shift(int N) { return N > 64 ? ilog2_host(N / 64) : 0; }

cudaError_t launch_sort(cudaStream_t s, int precision, const ParticleState& a, const ParticleState& b, int64_t n,
                        int64_t n_part, int n_species, int N, double L, uint32_t* key, uint32_t* hist,
                        uint32_t* bsum)
{
    if (n <= 0) return cudaSuccess;
    const int shift = sort_tile_shift(N);
    const uint32_t tpa = (uint32_t)(N >> shift);
    const uint32_t tiles = tpa * tpa * tpa;
    const int bins = (int)(tiles * (uint32_t)n_species);
    cudaError_t e = cudaMemsetAsync(hist, 0, (size_t)bins * 4, s);
    if (e != cudaSuccess) return e;
    const unsigned g = grid_for(n);
    if (precision == FDF_PREC_F64)
        k_sort_keys<FDF_PREC_F64><<<g, kThreads, 0, s>>>(a, n, n_part, (uint32_t)N, shift, tiles, N / L, key, hist);
    else
        k_sort_keys<FDF_PREC_F32><<<g, kThreads, 0, s>>>(a, n, n_part, (uint32_t)N, shift, tiles, N / L, key, hist);
    const int nb = (bins + 4 * kThreads - 1) / (4 * kThreads);
    k_scan_local<<<nb, kThreads, 0, s>>>(hist, hist, bsum, bins);
    k_scan_totals<<<1, kThreads, 0, s>>>(bsum, nb);
    k_scan_add<<<nb, kThreads, 0, s>>>(hist, bsum, bins);
    if (precision == FDF_PREC_F64) k_sort_scatter<FDF_PREC_F64><<<g, kThreads, 0, s>>>(a, b, n, key, hist);
    else k_sort_scatter<FDF_PREC_F32><<<g, kThreads, 0, s>>>(a, b, n, key, hist);
    return cudaGetLastError();
}

}  // namespace fdf
