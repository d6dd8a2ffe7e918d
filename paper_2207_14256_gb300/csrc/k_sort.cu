// k_sort.cu -- re-bucketing of particles by position for gather locality.
//
// Each particle's arithmetic is independent of the others (the metric is
// computed beforehand in linear theory, Sec. 2.1), so the particle arrays may
// be permuted freely; results are read back by particle id.  Particles are
// ordered by key = species * B + Morton(bucket), a bucket being a cube of
// 2^sort_tile cells per axis (B buckets per species) around the particle's
// predicted position halfway through the next pass, with a counting sort:
//   keys:    key of every particle and a histogram of keys;
//   scan:    exclusive prefix sum of the histogram (recursive, any bin count);
//   pack:    every particle's state, as one 64-byte record, goes to
//            offset[key]++ (warp-aggregated atomics, two particles in flight
//            per thread);
//   unpack:  the records go back to the arrays of the other half of the
//            double-buffered state.
// Within a bucket the order is whatever the atomics produce; no result
// depends on it.
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

template <int F>
__global__ void __launch_bounds__(kThreads) k_sort_keys(ParticleState st, int64_t n, int64_t n_part, uint32_t N,
                                                        int tile_shift, uint32_t tiles_per_species, double invh,
                                                        SortLead lead, uint32_t* __restrict__ key,
                                                        uint32_t* __restrict__ hist)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x; i0 < n; i0 += stride) {
        const int64_t i = i0 + threadIdx.x;
        const bool live = i < n;
        const unsigned active = __ballot_sync(0xffffffffu, live);
        if (!live) continue;
        const uint32_t s = (uint32_t)(i / n_part);
        uint32_t c[3];
        if constexpr (F == kPlain) {
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                int ci = (int)floor(st.xd[d * n + i] * invh);
                ci = ci < 0 ? 0 : (ci >= (int)N ? (int)N - 1 : ci);
                c[d] = (uint32_t)ci >> tile_shift;
            }
        } else if constexpr (F == kWide) {
            // the cell of x + q dtau / sqrt(q^2 + m^2 a^2) (the lead in cells), wrapped
            float q[3], q2 = 0.f;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                q[d] = (float)st.qd[d * n + i];
                q2 = fmaf(q[d], q[d], q2);
            }
            const float k = lead.on ? lead.dtau_q32[s] * ((float)N * 2.3283064365386963e-10f) *
                                          rsqrtf(q2 + lead.m2a2[s])
                                    : 0.f;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                float u = (float)st.xd[d * n + i] * (float)invh + q[d] * k;
                u = fminf(fmaxf(u, -1.0e6f), 1.0e6f);      // a saturated lead is only a poor guess
                int ci = (int)floorf(u) % (int)N;
                ci = ci < 0 ? ci + (int)N : ci;
                c[d] = (uint32_t)ci >> tile_shift;
            }
        } else {
            float q[3] = {0.f, 0.f, 0.f};
            float k = 0.f;
            if (lead.on) {   // without a lead the momenta are not read (they may not exist yet)
                float q2 = 0.f;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    q[d] = st.q0f[d * n + i] + st.dqf[d * n + i];
                    q2 = fmaf(q[d], q[d], q2);
                }
                k = lead.dtau_q32[s] * rsqrtf(q2 + lead.m2a2[s]);
            }
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                // a saturated shift only makes the bucket a poor guess, never wrong
                const float shift = fminf(fmaxf(q[d] * k, -2.0e9f), 2.0e9f);
                const uint32_t Xp = st.X[d * n + i] + (uint32_t)__float2int_rn(shift);
                c[d] = __umulhi(Xp, N) >> tile_shift;
            }
        }
        const uint32_t k = s * tiles_per_species + (spread3(c[0]) | (spread3(c[1]) << 1) | (spread3(c[2]) << 2));
        key[i] = k;
        // lanes with the same key (neighbours in a sorted state) add once through a leader
        const unsigned peers = __match_any_sync(active, k);
        if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(hist + k, (uint32_t)__popc(peers));
    }
}

// Exclusive scan, phase 1: each block scans 4 * kThreads elements and writes its total.
__global__ void __launch_bounds__(kThreads) k_scan_local(uint32_t* __restrict__ v, uint32_t* __restrict__ bsum,
                                                         int64_t n)
{
    __shared__ uint32_t warp_tot[kThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * 4 * kThreads + 4 * threadIdx.x;
    uint32_t x4[4], t = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        x4[j] = base + j < n ? v[base + j] : 0u;
        t += x4[j];
    }
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
    uint32_t run = x - t + (wid ? warp_tot[wid - 1] : 0u);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (base + j < n) v[base + j] = run;
        run += x4[j];
    }
    if (threadIdx.x == kThreads - 1) bsum[blockIdx.x] = run;
}

// Phase 3: add the scanned block totals.
__global__ void __launch_bounds__(kThreads) k_scan_add(uint32_t* __restrict__ v, const uint32_t* __restrict__ bsum,
                                                       int64_t n)
{
    const int64_t base = (int64_t)blockIdx.x * 4 * kThreads;
    const uint32_t add = bsum[blockIdx.x];
    for (int j = threadIdx.x; j < 4 * kThreads; j += kThreads)
        if (base + j < n) v[base + j] += add;
}

// Exclusive scan of v[0..n) in place; the totals of each level go to tmp.
cudaError_t scan_exclusive(cudaStream_t s, uint32_t* v, int64_t n, uint32_t* tmp)
{
    const int64_t per = 4 * kThreads;
    const int64_t nb = (n + per - 1) / per;
    k_scan_local<<<(unsigned)nb, kThreads, 0, s>>>(v, tmp, n);
    if (nb > 1) {
        cudaError_t e = scan_exclusive(s, tmp, nb, tmp + nb);
        if (e != cudaSuccess) return e;
        k_scan_add<<<(unsigned)nb, kThreads, 0, s>>>(v, tmp, n);
    }
    return cudaGetLastError();
}

// Scatter: every particle's state, packed into one record, goes to offset[key]++.
// Records keep the scattered writes whole (48 bytes instead of nine 4-byte fields).
struct alignas(64) SplitRec {   // 64 bytes: a scattered record covers two whole sectors
    uint32_t X[3];
    float q0[3];
    float dq[3];
    uint32_t id;
    double pmag;
    uint32_t pad[4];
};
struct alignas(32) PlainRec {   // 128 bytes: four whole sectors
    double x[3], q[3], q0[3], pmag, s;   // s: phi + psi of the exact equations of motion
    uint32_t id, pad[5];
};
static_assert(sizeof(PlainRec) == 128, "PlainRec is four sectors");

struct alignas(32) WideRec {    // 96 bytes: three whole sectors
    double x[3], q[3];
    float q0[3];
    uint32_t id;
    double pmag;
    uint32_t pad[4];
};
static_assert(sizeof(WideRec) == 96, "WideRec is three sectors");

template <int F> struct RecOf { using T = SplitRec; };
template <> struct RecOf<kPlain> { using T = PlainRec; };
template <> struct RecOf<kWide> { using T = WideRec; };

// A wide record moves as three 32-byte vector accesses (records are 32-byte aligned).
__device__ __forceinline__ void store_wide(void* recs, int64_t j, const WideRec& r)
{
    const uint32_t* w = reinterpret_cast<const uint32_t*>(&r);
    uint32_t* p = reinterpret_cast<uint32_t*>(recs) + 24 * j;
#pragma unroll
    for (int h = 0; h < 3; ++h)
        asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p + 8 * h), "r"(w[8 * h]),
                     "r"(w[8 * h + 1]), "r"(w[8 * h + 2]), "r"(w[8 * h + 3]), "r"(w[8 * h + 4]), "r"(w[8 * h + 5]),
                     "r"(w[8 * h + 6]), "r"(w[8 * h + 7])
                     : "memory");
}

__device__ __forceinline__ WideRec load_wide(const void* recs, int64_t j)
{
    WideRec r;
    uint32_t* w = reinterpret_cast<uint32_t*>(&r);
    const uint32_t* p = reinterpret_cast<const uint32_t*>(recs) + 24 * j;
#pragma unroll
    for (int h = 0; h < 3; ++h)
        asm volatile("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                     : "=r"(w[8 * h]), "=r"(w[8 * h + 1]), "=r"(w[8 * h + 2]), "=r"(w[8 * h + 3]), "=r"(w[8 * h + 4]),
                       "=r"(w[8 * h + 5]), "=r"(w[8 * h + 6]), "=r"(w[8 * h + 7])
                     : "l"(p + 8 * h));
    return r;
}

// A split record moves as two 32-byte vector accesses (the record buffer and each
// record are 64-byte aligned).
__device__ __forceinline__ void store_split(void* recs, int64_t j, const SplitRec& r)
{
    uint32_t* p = reinterpret_cast<uint32_t*>(recs) + 16 * j;
    asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(r.X[0]), "r"(r.X[1]),
                 "r"(r.X[2]), "r"(__float_as_uint(r.q0[0])), "r"(__float_as_uint(r.q0[1])),
                 "r"(__float_as_uint(r.q0[2])), "r"(__float_as_uint(r.dq[0])), "r"(__float_as_uint(r.dq[1]))
                 : "memory");
    asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p + 8),
                 "r"(__float_as_uint(r.dq[2])), "r"(r.id), "r"((uint32_t)__double2loint(r.pmag)),
                 "r"((uint32_t)__double2hiint(r.pmag)), "r"(0u), "r"(0u), "r"(0u), "r"(0u)
                 : "memory");
}

__device__ __forceinline__ SplitRec load_split(const void* recs, int64_t j)
{
    const uint32_t* p = reinterpret_cast<const uint32_t*>(recs) + 16 * j;
    uint32_t w[16];
    asm volatile("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7])
                 : "l"(p));
    asm volatile("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(w[8]), "=r"(w[9]), "=r"(w[10]), "=r"(w[11]), "=r"(w[12]), "=r"(w[13]), "=r"(w[14]),
                   "=r"(w[15])
                 : "l"(p + 8));
    SplitRec r;
    for (int d = 0; d < 3; ++d) {
        r.X[d] = w[d];
        r.q0[d] = __uint_as_float(w[3 + d]);
        r.dq[d] = __uint_as_float(w[6 + d]);
    }
    r.id = w[9];
    r.pmag = __hiloint2double((int)w[11], (int)w[10]);
    r.pad[0] = r.pad[1] = r.pad[2] = r.pad[3] = 0;
    return r;
}

template <int F>
__device__ __forceinline__ void make_rec(const ParticleState& a, int64_t n, int64_t i, typename RecOf<F>::T& r,
                                         bool pre_transform = false)
{
    if constexpr (F == kWide) {
        for (int d = 0; d < 3; ++d) {
            r.x[d] = a.xd[d * n + i];
            r.q[d] = a.qd[d * n + i];
            r.q0[d] = a.q0f[d * n + i];
        }
        r.id = a.id[i];
        r.pmag = a.pmag[i];
        for (int q = 0; q < 4; ++q) r.pad[q] = 0;
    } else if constexpr (F == kPlain) {
        for (int d = 0; d < 3; ++d) {
            r.x[d] = a.xd[d * n + i];
            r.q[d] = a.qd[d * n + i];
            r.q0[d] = a.q0d[d * n + i];
        }
        r.pmag = a.pmag[i];
        r.s = a.sd ? a.sd[i] : 0.0;
        r.id = a.id[i];
        for (int q = 0; q < 5; ++q) r.pad[q] = 0;
    } else {
        for (int d = 0; d < 3; ++d) r.X[d] = a.X[d * n + i];
        if (pre_transform) {
            // the three FP64 sampled momenta, bit for bit, in the six 32-bit momentum slots
            uint32_t w[6];
            for (int d = 0; d < 3; ++d) {
                const double v = a.qs[d * n + i];
                w[2 * d] = (uint32_t)__double2loint(v);
                w[2 * d + 1] = (uint32_t)__double2hiint(v);
            }
            for (int d = 0; d < 3; ++d) {
                r.q0[d] = __uint_as_float(w[d]);
                r.dq[d] = __uint_as_float(w[3 + d]);
            }
        } else {
            for (int d = 0; d < 3; ++d) {
                r.q0[d] = a.q0f[d * n + i];
                r.dq[d] = a.dqf[d * n + i];
            }
        }
        r.id = a.id[i];
        r.pmag = a.pmag[i];
        r.pad[0] = r.pad[1] = r.pad[2] = r.pad[3] = 0;
    }
}

// Each thread takes kPackU particles per trip and issues all their offset atomics
// before it waits for any: the keys of a warp are mostly distinct, so an atomic's
// round trip to L2 is what a particle waits for, and kPackU of them overlap.
constexpr int kPackU = 2;

template <int F>
__global__ void __launch_bounds__(kThreads) k_sort_pack(ParticleState a, int64_t n, const uint32_t* __restrict__ key,
                                                        uint32_t* __restrict__ offset, void* __restrict__ recs,
                                                        int pre_transform)
{
    using Rec = typename RecOf<F>::T;
    // Grid-stride loop with a warp-uniform trip count, so that every lane can take
    // part in the warp-aggregated atomics: lanes sharing a key take one atomicAdd
    // through their leader.
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x; i0 < n; i0 += kPackU * stride) {
        int64_t idx[kPackU];
        uint32_t k[kPackU], base[kPackU];
        unsigned peers[kPackU];
        int leader[kPackU];
        bool live[kPackU];
        Rec r[kPackU];
#pragma unroll
        for (int u = 0; u < kPackU; ++u) {
            idx[u] = i0 + u * stride + threadIdx.x;
            live[u] = idx[u] < n;
            k[u] = live[u] ? key[idx[u]] : 0u;
            base[u] = 0u;
            if (live[u]) make_rec<F>(a, n, idx[u], r[u], pre_transform != 0);
        }
#pragma unroll
        for (int u = 0; u < kPackU; ++u) {
            const unsigned active = __ballot_sync(0xffffffffu, live[u]);
            peers[u] = 0u;
            leader[u] = 0;
            if (live[u]) {
                peers[u] = __match_any_sync(active, k[u]);
                leader[u] = __ffs(peers[u]) - 1;
                if (lane == leader[u]) base[u] = atomicAdd(offset + k[u], (uint32_t)__popc(peers[u]));
            }
        }
#pragma unroll
        for (int u = 0; u < kPackU; ++u) {
            if (!live[u]) continue;
            const uint32_t b = __shfl_sync(peers[u], base[u], leader[u]);
            const int64_t j = (int64_t)b + __popc(peers[u] & ((1u << lane) - 1u));
            if constexpr (F == kPlain) reinterpret_cast<Rec*>(recs)[j] = r[u];
            else if constexpr (F == kWide) store_wide(recs, j, r[u]);
            else store_split(recs, j, r[u]);
        }
    }
}

template <int F>
__global__ void __launch_bounds__(kThreads) k_sort_unpack(ParticleState b, int64_t n, const void* __restrict__ recs,
                                                          int pre_transform)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        if constexpr (F == kWide) {
            const WideRec r = load_wide(recs, j);
            for (int d = 0; d < 3; ++d) {
                b.xd[d * n + j] = r.x[d];
                b.qd[d * n + j] = r.q[d];
                b.q0f[d * n + j] = r.q0[d];
            }
            b.pmag[j] = r.pmag;
            b.id[j] = r.id;
        } else if constexpr (F == kPlain) {
            const PlainRec r = reinterpret_cast<const PlainRec*>(recs)[j];
            for (int d = 0; d < 3; ++d) {
                b.xd[d * n + j] = r.x[d];
                b.qd[d * n + j] = r.q[d];
                b.q0d[d * n + j] = r.q0[d];
            }
            b.pmag[j] = r.pmag;
            if (b.sd) b.sd[j] = r.s;
            b.id[j] = r.id;
        } else {
            const SplitRec r = load_split(recs, j);
            for (int d = 0; d < 3; ++d) b.X[d * n + j] = r.X[d];
            if (pre_transform) {
                // the sampled momenta (one array shared by both halves: the pack kernel
                // has read all of it before this kernel writes)
                uint32_t w[6];
                for (int d = 0; d < 3; ++d) {
                    w[d] = __float_as_uint(r.q0[d]);
                    w[3 + d] = __float_as_uint(r.dq[d]);
                }
                for (int d = 0; d < 3; ++d) b.qs[d * n + j] = __hiloint2double((int)w[2 * d + 1], (int)w[2 * d]);
            } else {
                for (int d = 0; d < 3; ++d) {
                    b.q0f[d * n + j] = r.q0[d];
                    b.dqf[d * n + j] = r.dq[d];
                }
            }
            b.id[j] = r.id;
            b.pmag[j] = r.pmag;
        }
    }
}

// ---- export in id order through the record buffer -------------------------------
// A sorted state holds particle i's outputs at slot id[i] - begin of the caller's
// arrays.  Writing them there directly scatters seven 8-byte values per particle;
// instead each particle's record goes whole to that slot (one scattered 64-byte
// write), and a streaming pass turns the records into positions, momenta and
// weights.
template <int F>
__global__ void __launch_bounds__(kThreads) k_export_pack(ParticleState a, int64_t n, int64_t begin, int64_t count,
                                                          void* __restrict__ recs)
{
    using Rec = typename RecOf<F>::T;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < count;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = begin + j;
        const int64_t o = (int64_t)a.id[i] - begin;
        Rec r;
        make_rec<F>(a, n, i, r);
        if constexpr (F == kPlain) reinterpret_cast<Rec*>(recs)[o] = r;
        else if constexpr (F == kWide) store_wide(recs, o, r);
        else store_split(recs, o, r);
    }
}

template <int F>
__global__ void __launch_bounds__(kThreads) k_export_unpack(const void* __restrict__ recs, int64_t count, double L,
                                                            double T, double* __restrict__ xo,
                                                            double* __restrict__ qo, double* __restrict__ wo)
{
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < count;
         o += (int64_t)gridDim.x * blockDim.x) {
        double x[3], q[3], pm;
        if constexpr (F == kWide) {
            const WideRec r = load_wide(recs, o);
            for (int d = 0; d < 3; ++d) {
                x[d] = r.x[d];
                q[d] = r.q[d];
            }
            pm = r.pmag;
        } else if constexpr (F == kPlain) {
            const PlainRec r = reinterpret_cast<const PlainRec*>(recs)[o];
            for (int d = 0; d < 3; ++d) {
                x[d] = r.x[d];
                q[d] = r.q[d];
            }
            pm = r.pmag;
        } else {
            const SplitRec r = load_split(recs, o);
            for (int d = 0; d < 3; ++d) {
                x[d] = L * ((double)r.X[d] * 2.3283064365386963e-10);
                q[d] = (double)r.q0[d] + (double)r.dq[d];
            }
            pm = r.pmag;
        }
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
            if constexpr (F == kPlain) wo[o] = dfweight(norm3_rn(q), pm, T);
            else wo[o] = (double)dfweight_split(norm3_rn(q), pm, T);
        }
    }
}

unsigned grid_for(int64_t n)
{
    int64_t b = (n + kThreads - 1) / kThreads;
    if (b > 152 * 16) b = 152 * 16;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

size_t sort_record_bytes(int precision)
{
    const int f = form_of(precision);
    // the FP64-state form also sorts once before the transform, with split records
    return f == kPlain ? sizeof(PlainRec) : f == kWide ? sizeof(WideRec) : sizeof(SplitRec);
}

cudaError_t launch_sort(cudaStream_t s, int precision, const ParticleState& a, const ParticleState& b, int64_t n,
                        int64_t n_part, int n_species, int N, int tile_shift, double L, const SortLead& lead,
                        uint32_t* key, uint32_t* hist, uint32_t* bsum, void* recs)
{
    if (n <= 0) return cudaSuccess;
    const int shift = tile_shift;
    const uint32_t tpa = (uint32_t)(N >> shift);
    const uint32_t tiles = tpa * tpa * tpa;
    const int64_t bins = (int64_t)tiles * n_species;
    cudaError_t e = cudaMemsetAsync(hist, 0, (size_t)bins * 4, s);
    if (e != cudaSuccess) return e;
    const unsigned g = grid_for(n);
    // Before the momentum transform the FP64-state and split-state forms hold the
    // sampler's output only (fixed-point positions, sampled momenta): both sort it as
    // the split-state form does.
    int f = form_of(precision);
    if (lead.pre_transform) f = kFixed;
#define FDF_SORT(F_)                                                                                                  \
    do {                                                                                                              \
        k_sort_keys<F_><<<g, kThreads, 0, s>>>(a, n, n_part, (uint32_t)N, shift, tiles, N / L, lead, key, hist);     \
        e = scan_exclusive(s, hist, bins, bsum);                                                                      \
        if (e != cudaSuccess) return e;                                                                               \
        k_sort_pack<F_><<<g, kThreads, 0, s>>>(a, n, key, hist, recs, lead.pre_transform);                           \
        k_sort_unpack<F_><<<g, kThreads, 0, s>>>(b, n, recs, lead.pre_transform);                                    \
    } while (0)
    if (f == kPlain) FDF_SORT(kPlain);
    else if (f == kWide) FDF_SORT(kWide);
    else FDF_SORT(kFixed);
#undef FDF_SORT
    return cudaGetLastError();
}

cudaError_t launch_export_records(cudaStream_t s, int precision, const ParticleState& st, int64_t n, int64_t begin,
                                  int64_t count, double L, double T_ev, void* recs, double* x, double* q, double* w)
{
    if (count <= 0) return cudaSuccess;
    const unsigned b = grid_for(count);
    const int f = form_of(precision);
#define FDF_EXPORT(F_)                                                                                                \
    do {                                                                                                              \
        k_export_pack<F_><<<b, kThreads, 0, s>>>(st, n, begin, count, recs);                                          \
        k_export_unpack<F_><<<b, kThreads, 0, s>>>(recs, count, L, T_ev, x, q, w);                                    \
    } while (0)
    if (f == kPlain) FDF_EXPORT(kPlain);
    else if (f == kWide) FDF_EXPORT(kWide);
    else FDF_EXPORT(kFixed);
#undef FDF_EXPORT
    return cudaGetLastError();
}

}  // namespace fdf
