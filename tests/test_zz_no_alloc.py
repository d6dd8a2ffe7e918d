"""fdf_build_fields_noalloc against fdf_build_fields.

The no-alloc entry point exists for callers that must not allocate device
memory (an embedding simulation whose allocator owns the device budget, or a
serving loop that forbids cudaMalloc/cudaFree after start-up).  It runs the
same field kernels with their work arrays in a static device array, so its
output must equal the context path's.  Two calls in a row check that the
shared array, which keeps the previous call's contents, does not leak into the
next result.  This file sorts last so that a run stopping at the first failure
has already run every other test.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

TOL_F32_FIELDS = 3e-6   # the FP32 field tolerance of the parity tests


@pytest.fixture(scope="module")
def F():
    from paper_2207_14256_gb300 import build
    from paper_2207_14256_gb300 import fdf

    build.build()
    fdf.lib()
    return fdf


def test_noalloc_fields_equal_context_fields_on_two_calls(F, inputs, c1_tables):
    import torch

    p = inputs.config("c1_32", n_grid=32, precision=1, seed=31)
    o = O.Oracle(p, c1_tables)
    lnas = [o.lna(37), o.lna(100)]
    with F.Run(p, c1_tables) as r:
        refs = [r.build_fields(l) for l in lnas]
    P = F.make_params(p)
    T, keep = F.make_tables(c1_tables)
    N = p["n_grid"]
    out = torch.empty((8, N, N, N), dtype=torch.float64, device="cuda")
    for lna, ref in zip(lnas, refs):
        out.fill_(float("nan"))
        F.fdf_build_fields_noalloc(P, T, lna, out)
        got = out.cpu().numpy()
        for s in range(8):
            pair = s & ~1   # slots are transformed in packed pairs (see the parity tests)
            scale = max(np.max(np.abs(ref[pair])), np.max(np.abs(ref[pair + 1])))
            err = np.max(np.abs(got[s] - ref[s])) / scale
            print("lna %.3f slot %d: max |noalloc - context| / scale = %.3e" % (lna, s, err))
            assert err <= TOL_F32_FIELDS


def test_noalloc_rejects_grids_beyond_the_scratch(F, inputs, c1_tables):
    import torch

    P = F.make_params(inputs.config("c1_32", n_grid=128, precision=1))
    T, keep = F.make_tables(c1_tables)
    out = torch.empty(8, dtype=torch.float64, device="cuda")
    with pytest.raises(F.FdfError) as e:
        F.fdf_build_fields_noalloc(P, T, -10.0, out)
    assert e.value.code == F.FDF_EINVAL
    assert "FDF_NOALLOC_SCRATCH_BYTES" in F.fdf_last_error()
