// fields_noalloc.cu -- fdf_build_fields_noalloc: the field build of
// fdf_build_fields without a context and without any device allocation.
//
// Some callers cannot allocate device memory: a simulation code that embeds
// this library and whose own allocator owns the whole device budget, or a
// serving loop that forbids cudaMalloc/cudaFree after start-up because those
// calls synchronise the device and fragment its memory.  This entry point
// serves them.  Its work arrays live in one file-scope device array of
// FDF_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until the
// process exits; the caller passes the inputs (host tables) and the output
// (device memory).
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "device_math.cuh"

namespace fdf {
namespace {

// The shared scratch.  Host code must not pass g_scratch itself to a kernel:
// in host code the name is a host-side stand-in, not a device address.  Its
// device address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_scratch[FDF_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Device address of g_scratch on the current device; looked up on the first
// call made with that device current.
int scratch_address(unsigned char** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(FDF_ECUDA, (std::string("cudaGetDevice: ") + cudaGetErrorString(e)).c_str());
    if (dev < 0 || dev >= kMaxDevices) return set_error(FDF_ENOSYS, "device index beyond 63");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p)
            return set_error(FDF_ECUDA, (std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e)).c_str());
        g_scratch_addr[dev] = p;
    }
    *out = (unsigned char*)g_scratch_addr[dev];
    return FDF_OK;
}

}  // namespace
}  // namespace fdf

using namespace fdf;

extern "C" int fdf_build_fields_noalloc(const fdf_params* p, const fdf_tables* t, double lna, double* out,
                                        void* stream)
{
    int rc = validate_params(p);
    if (rc) return rc;
    if (!t || !t->lnk || !t->lna || !t->T_psi || !t->T_phi || !t->dTphi_dlna || !out || !std::isfinite(lna))
        return set_error(FDF_EINVAL, "bad arguments");
    if (t->nk < 2 || t->na < 2 || t->nk > 1024 || t->na > 256)
        return set_error(FDF_EINVAL, "table sizes out of range (nk 2..1024, na 2..256)");
    double lnk0, dlnk, lnat0, dlnat;
    if (!uniform_grid(t->lnk, t->nk, &lnk0, &dlnk) || !uniform_grid(t->lna, t->na, &lnat0, &dlnat))
        return set_error(FDF_EINVAL, "lnk and lna must be uniform ascending grids");
    const int gp = grid_prec(p->precision);
    const bool f64 = gp == FDF_PREC_F64;
    const size_t N = (size_t)p->n_grid, N3 = N * N * N;
    const size_t csz = f64 ? 16 : 8, rsz = f64 ? 8 : 4;
    const size_t ntab = 3 * (size_t)t->na * t->nk;
    // scratch layout: W0 | W1 | FP64 tables | amplitude table | twiddles | noise; the
    // interleaved grid G of the last pass reuses W0 (same size or smaller).
    const size_t M = (size_t)mode_table_size(p->n_grid);
    const size_t oW0 = 0, oW1 = oW0 + align256(4 * N3 * csz), oT64 = oW1 + align256(4 * N3 * csz);
    const size_t oA = oT64 + align256(ntab * 8), oTw = oA + align256(4 * M * rsz), oR = oTw + align256(N * csz);
    const size_t need = oR + align256(N3 * csz);
    if (need > FDF_NOALLOC_SCRATCH_BYTES) {
        char msg[200];
        snprintf(msg, sizeof msg,
                 "fdf_build_fields_noalloc: n_grid %d at this precision needs %zu bytes of scratch; the static "
                 "scratch holds %zu (FDF_NOALLOC_SCRATCH_BYTES)",
                 p->n_grid, need, (size_t)FDF_NOALLOC_SCRATCH_BYTES);
        return set_error(FDF_EINVAL, msg);
    }
    unsigned char* s = nullptr;
    rc = scratch_address(&s);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nt = (size_t)t->na * t->nk;
    double* T64 = (double*)(s + oT64);
    cudaError_t e = cudaMemcpyAsync(T64, t->T_psi, nt * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(T64 + nt, t->T_phi, nt * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(T64 + 2 * nt, t->dTphi_dlna, nt * 8, cudaMemcpyHostToDevice, st);
    // the twiddles fdf_create uploads, from the same host table; the copies are from
    // pageable host memory, so the stream is synchronised before the vectors go
    std::vector<double> twd(2 * N);
    twiddle_table((int)N, twd.data());
    const std::vector<float> twf(twd.begin(), twd.end());
    if (e == cudaSuccess)
        e = f64 ? cudaMemcpyAsync(s + oTw, twd.data(), twd.size() * 8, cudaMemcpyHostToDevice, st)
                : cudaMemcpyAsync(s + oTw, twf.data(), twf.size() * 4, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return set_error(FDF_ECUDA, (std::string("table upload: ") + cudaGetErrorString(e)).c_str());
    FieldArgs a = make_field_args(*p, t->nk, t->na, lnk0, dlnk, lnat0, dlnat, lna);
    void* W0 = s + oW0;
    void* W1 = s + oW1;
    if (e == cudaSuccess) e = launch_noise(st, gp, a, s + oR);
    if (e == cudaSuccess) e = launch_mode_table(st, gp, a, T64, s + oA);
    // as fdf_build_fields: slots 0-6 from a build with phi_dot transformed alone, slot 7
    // (psi) from a second build
    for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {
        a.slot7 = pass == 0 ? kSlot7Zero : kSlot7Psi;
        e = launch_fields_z(st, gp, a, s + oA, s + oR, s + oTw, W0);
        if (e == cudaSuccess) e = launch_fields_y(st, gp, a, s + oTw, W0, W1);
        if (e == cudaSuccess) e = launch_fields_x(st, gp, a, s + oTw, W1, W0);
        if (e == cudaSuccess) e = launch_fields_to_f64(st, gp, p->n_grid, W0, out, pass == 0 ? 0x7Fu : 0x80u);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess)
        return set_error(FDF_ECUDA, (std::string("fdf_build_fields_noalloc: ") + cudaGetErrorString(e)).c_str());
    return FDF_OK;
}
