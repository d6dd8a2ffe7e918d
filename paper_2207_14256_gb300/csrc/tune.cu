// tune.cu -- fdf_tune: the autotuner of the schedule knobs.
//
// Five knobs change the speed of a run but not its results beyond the stated
// tolerances: how far particles may drift before they are re-bucketed
// (sort_cells), the size of a bucket (sort_tile: cubes of 2^t cells per axis),
// the number of leapfrog steps one particle pass covers (steps_per_pass) and, for
// the FP64-state forms, the launch shape of the pass (pass_blocks), for the
// split-state forms, whether kicks read the grid from shared-memory tiles (gather_tile).
// Their best values depend on the workload: on how fast the particles cross
// cells (mass, momentum, box, step), on the grid size against L2 and on the
// particle count.  The tuner times whole runs on the device and walks the knobs
// one at a time from the automatic choices (coordinate descent).
#include <cmath>
#include <string>
#include <vector>

#include "fdf_internal.cuh"

namespace fdf {
namespace {

// One timed run of q: fdf_sample + fdf_step(n_steps), CUDA events on the stream.
int timed_run(const fdf_params& q, const fdf_tables* t, cudaStream_t s, double* ms)
{
    fdf_ctx* c = nullptr;
    int rc = fdf_create(&q, t, s, nullptr, 0, &c);
    if (rc) return rc;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) {
        rc = fdf_sample(c);
        if (!rc) rc = fdf_step(c, q.n_steps);
        if (!rc) e = cudaEventRecord(e1, s);
        if (!rc && e == cudaSuccess) e = cudaEventSynchronize(e1);
        float f = 0.f;
        if (!rc && e == cudaSuccess) e = cudaEventElapsedTime(&f, e0, e1);
        *ms = f;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    fdf_destroy(c);
    if (!rc && e != cudaSuccess) rc = set_error(FDF_ECUDA, (std::string("fdf_tune: ") + cudaGetErrorString(e)).c_str());
    return rc;
}

}  // namespace
}  // namespace fdf

using namespace fdf;

extern "C" int fdf_tune(const fdf_params* p, const fdf_tables* t, void* stream, fdf_params* out, double* ms,
                        int32_t* trials)
{
    if (!p || !t || !out) return set_error(FDF_EINVAL, "NULL argument");
    int rc = validate_params(p);
    if (rc) return rc;
    *out = *p;
    if (trials) *trials = 0;
    if (ms) *ms = 0;
    if (p->precision == FDF_PREC_F64 || p->n_part == 0) return FDF_OK;
    cudaStream_t s = (cudaStream_t)stream;
    fdf_params best = *p;
    best.sort_every = 0;
    best.sort_cells = 4;
    best.sort_tile = 0;
    best.steps_per_pass = 4;
    const bool wide = form_of(p->precision) == kWide;
    best.pass_blocks = wide ? 2 : 0;
    best.gather_tile = wide ? 0 : -1;
    double best_ms = 0;
    int n = 0;
    // one untimed run first (module load, first-touch of the allocation)
    rc = timed_run(best, t, s, &best_ms);
    if (rc) return rc;
    rc = timed_run(best, t, s, &best_ms);
    if (rc) return rc;
    ++n;
    struct Knob {
        int32_t fdf_params::*field;
        std::vector<int32_t> values;
    };
    // a coarse pass over each knob, then the re-sort distance again between the coarse
    // values (its best value moves with the bucket size chosen after it)
    const std::vector<Knob> knobs = {{&fdf_params::sort_cells, {2, 4, 8, 16, 32, 64}},
                                     {&fdf_params::sort_tile, {0, 1, 2, 3}},
                                     {&fdf_params::steps_per_pass, {2, 3, 4, 6, 8}},
                                     {&fdf_params::pass_blocks, {2, 3}},
                                     {&fdf_params::gather_tile, {-1, 1}},
                                     {&fdf_params::sort_cells, {3, 5, 6, 12, 24, 48}}};
    for (const Knob& k : knobs) {
        if (k.field == &fdf_params::pass_blocks && !wide) continue;
        if (k.field == &fdf_params::gather_tile && wide) continue;
        const int32_t start = best.*(k.field);
        for (int32_t v : k.values) {
            if (v == start) continue;
            fdf_params q = best;
            q.*(k.field) = v;
            if (q.sort_tile > 0 && (q.n_grid >> q.sort_tile) < 1) continue;
            double m = 0;
            rc = timed_run(q, t, s, &m);
            if (rc) return rc;
            ++n;
            if (m < best_ms) {
                best_ms = m;
                best = q;
            }
        }
    }
    *out = best;
    if (ms) *ms = best_ms;
    if (trials) *trials = n;
    return FDF_OK;
}
